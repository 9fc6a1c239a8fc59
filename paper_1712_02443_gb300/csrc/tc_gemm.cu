// Tensor-core (tcgen05) form of the macromodel contraction, BF16 or FP16 inputs
// with FP32 accumulation in tensor memory (Sec. III / eq. (MV_product1): the
// per-type products u = M x, v = D x of identical elements).
//
// The complex product is a real GEMM with interleaved real/imaginary rows:
//   A (4 Nh x 2 Nh): row 2i = [Re W_i, -Im W_i], row 2i+1 = [Im W_i, Re W_i]
//                    (W = [M; D] stacked, so i runs over 2 Nh output rows);
//   B (ncols x 2 Nh): column (element, rhs) = [Re x_e, Im x_e];
//   C = A B^T: row 2i = Re out_i, row 2i+1 = Im out_i.
// Both operands are K-major in global memory; A is padded to the tile with
// zeros, B is read through a tensor map whose out-of-range box entries are
// zero-filled by the copy engine.
//
// K is laid out as [Re part: Nh entries | zeros up to Nhp = Nh rounded up to 8 |
// Im part: Nh entries], so that both halves of a B row start 16-byte aligned.
//
// Kernel: persistent, one CTA per SM, 320 threads in three roles.
//   warp 0     one lane issues TMA copies of the 128 x 64 A slice and the
//              256 x 64 B slice of each k step into a 4-stage ring of
//              128-byte-swizzled K-major buffers;
//   warp 1     allocates 512 TMEM columns; one lane issues tcgen05.mma
//              (M 128, N 256, K 16) and commits each stage back to its slot;
//   warps 2-9  epilogue: tcgen05.ld of the accumulator (each warp reads the
//              TMEM lane quarter warp % 4 and one half of the columns), Re/Im
//              pairing through a shared staging tile, column-per-lane stores
//              of complex rows to u (rows < Nh) or v.
// Two accumulators (2 x 256 columns) let the epilogue of one tile overlap the
// main loop of the next.  Tiles are ordered M-fastest so that the CTAs working
// at one time share their B slices in L2.  Each CTA copies its own operands
// from this GPU's memory into its own shared memory (no cluster launch).
// Every mbarrier wait is bounded in time; on expiry the kernel
// records an error, the other roles stop, copies and products in flight are
// waited for (bounded) and TMEM is freed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <mutex>

#include "tc_gemm.h"
#include "tcgen05.cuh"

namespace mm {

namespace {

constexpr int TBM = 128, TBN = 256, TBK = 64, STAGES = 4;
constexpr int A_BYTES = TBM * TBK * 2;   // 16 KB
constexpr int B_BYTES = TBN * TBK * 2;   // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t kTmemCols = 2 * TBN;
constexpr int kThreads = 320;   // producer warp, MMA warp, 8 epilogue warps
constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s per wait (default limit)
constexpr unsigned long long kDrainNs = 1000000000ull;  // 1 s for copies / products in flight at exit

using namespace tcx;

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) { return make_desc_sw128(saddr); }

}  // namespace

// C (Mp x Np, FP32) = A (Mp x Kp) B^T (Np x Kp); epilogue writes complex rows
// (2i, 2i+1) of C to out_u (i < Nh) or out_v (i >= Nh) for column n = j*nrhs+c.
// wait_ns bounds every wait of the main loops; stall != 0 (a testing hook) makes
// the MMA issuer issue nothing, so that the other roles' waits run out.
template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int num_m,
              int num_groups, int nk, int Nh, int ncols, int nrhs, const int32_t* __restrict__ elems,
              const int64_t* __restrict__ off, float2* __restrict__ out_u, float2* __restrict__ out_v,
              int* __restrict__ err, uint64_t wait_ns, int stall) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2], tempty_bar[2], drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  volatile int* stop = &abort_flag;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // tiles g = (n tile) * num_m + (m tile), M fastest
  const int cid = blockIdx.x, ncl = gridDim.x;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull_bar[b]), 1);
      mbar_init(smem_u32(&tempty_bar[b]), 8);   // one arrival per epilogue warp
    }
    mbar_init(smem_u32(&drain_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer
      uint32_t it = 0;
      bool ok = true;
      for (int g = cid; g < num_groups && ok; g += ncl) {
        const int m0 = (g % num_m) * TBM, n0 = (g / num_m) * TBN;
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t r = it / STAGES;
          if (!mbar_wait(smem_u32(&empty_bar[s]), (r & 1) ^ 1, stop, wait_ns)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[s]);
          unsigned char* sa = base + s * STAGE_BYTES;
          mbar_expect_tx(fb, STAGE_BYTES);
          tma_load_2d(&tmA, smem_u32(sa), fb, kt * TBK, m0);
          tma_load_2d(&tmB, smem_u32(sa + A_BYTES), fb, kt * TBK, n0);
        }
      }
      if (!ok && !*stop) {
        *stop = 1;
        atomicExch(err, 1);
      }
      // copies still in flight land before the CTA's shared memory is released
      for (uint32_t q = it > (uint32_t)STAGES ? it - STAGES : 0; q < it; ++q)
        mbar_wait(smem_u32(&full_bar[q % STAGES]), (q / STAGES) & 1, nullptr, kDrainNs);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      constexpr uint32_t idesc = make_idesc(BF16 ? 1u : 0u, TBM, TBN);
      uint32_t it = 0, lt = 0;
      bool ok = true;
      for (int g = stall ? num_groups : cid; g < num_groups && ok; g += ncl, ++lt) {
        const uint32_t b = lt & 1, ub = lt >> 1;
        if (!mbar_wait(smem_u32(&tempty_bar[b]), (ub & 1) ^ 1, stop, wait_ns)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + b * TBN;
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t r = it / STAGES;
          if (!mbar_wait(smem_u32(&full_bar[s]), r & 1, stop, wait_ns)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(base + s * STAGE_BYTES);
          const uint64_t da = make_desc(sa), db = make_desc(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < TBK / 16; ++kk) {
            const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
            const uint64_t a = da + (uint64_t)((kk * 32) >> 4), bb = db + (uint64_t)((kk * 32) >> 4);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                "l"(a), "l"(bb), "r"(idesc), "r"(acc));
          }
          umma_commit(smem_u32(&empty_bar[s]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&tfull_bar[b]));
      }
      if (!ok && !*stop) {
        *stop = 1;
        atomicExch(err, 1);
      }
      // every product issued here completes before TMEM and the stage buffers go away
      umma_commit(smem_u32(&drain_bar));
      mbar_wait(smem_u32(&drain_bar), 0, nullptr, kDrainNs);
    }
  } else {
    // ---- epilogue (warps 2-9).  Warp w reads TMEM lane quarter q = w % 4 (C
    // rows m0 + 32q .. +31, complex rows i0 .. i0+15) and column half
    // (w - 2) / 4 of the accumulator.  Per 16-column chunk: TMEM -> registers
    // (lane = C row) -> shared staging [16 complex rows][16 columns] (row
    // stride 17 float2: the Re/Im writes of the 32 lanes fall in 32 distinct
    // banks) -> global, lanes 0-15 / 16-31 take one column each of two
    // consecutive rows, so a store instruction covers runs of consecutive
    // right-hand sides of one or more elements.
    const int q = warp & 3, half = (warp - 2) >> 2;
    float2* stage = reinterpret_cast<float2*>(base + STAGES * STAGE_BYTES) + (warp - 2) * (16 * 17);
    float* stage_f = reinterpret_cast<float*>(stage);
    constexpr int NCH = TBN / 2 / 16;   // 16-column chunks per warp
    const int col = lane & 15, rsub = lane >> 4;
    uint32_t lt = 0;
    bool ok = true;
    for (int g = cid; g < num_groups; g += ncl, ++lt) {
      const uint32_t b = lt & 1, ub = lt >> 1;
      const int m0 = (g % num_m) * TBM;
      const int nw = (g / num_m) * TBN + half * (TBN / 2);   // first column of this warp
      // output offsets of this lane's column in each chunk, loaded while the
      // accumulator is still being computed
      int64_t eb[NCH];
      int ccol[NCH];
#pragma unroll
      for (int k = 0; k < NCH; ++k) {
        const int n = nw + 16 * k + col;
        const int je = n < ncols ? n / nrhs : 0;
        ccol[k] = n < ncols ? n - je * nrhs : -1;
        eb[k] = elems[je];
      }
#pragma unroll
      for (int k = 0; k < NCH; ++k) eb[k] = off[eb[k]];
      int w_ok = 1;
      if (lane == 0) w_ok = mbar_wait(smem_u32(&tfull_bar[b]), ub & 1, stop, wait_ns) ? 1 : 0;
      w_ok = __shfl_sync(0xffffffffu, w_ok, 0);
      if (!w_ok) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int i0 = (m0 + 32 * q) >> 1;        // first complex output row of this warp
      const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + b * TBN + half * (TBN / 2);
#pragma unroll
      for (int k = 0; k < NCH; ++k) {
        uint32_t r[16];
        tmem_ld16(tbase + 16 * k, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // lane = C row 2*(lane/2) + (lane&1): Re (even) or Im (odd) of complex row lane/2
#pragma unroll
        for (int c = 0; c < 16; ++c) stage_f[(lane >> 1) * 34 + 2 * c + (lane & 1)] = __uint_as_float(r[c]);
        __syncwarp();
        const int cc = ccol[k];
        if (cc >= 0) {
          const int64_t e_base = eb[k];
#pragma unroll
          for (int it = 0; it < 8; ++it) {
            const int rr = 2 * it + rsub, i = i0 + rr;
            if (i < 2 * Nh) {
              const float2 val = stage[rr * 17 + col];
              if (i < Nh)
                out_u[(e_base + i) * nrhs + cc] = val;
              else
                out_v[(e_base + i - Nh) * nrhs + cc] = val;
            }
          }
        }
        __syncwarp();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[b]));
    }
    if (!ok && lane == 0 && !*stop) {
      *stop = 1;
      atomicExch(err, 1);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// B operand rows: row n = (element elems[n / nrhs], rhs n % nrhs) holds
// Re x_e(:, rhs) at [0, Nh) and Im x_e(:, rhs) at [Nhp, Nhp + Nh), 16-bit
// floats (entries outside are not written: A is zero there and the tensor map
// ends at Nhp + Nh).  Thread (element j, rhs c, row group g) reads rows
// 8g .. 8g+7 of x_e(:, c) (eight independent loads; consecutive threads take
// consecutive right-hand sides, so each load instruction uses whole sectors)
// and writes them as one 16-byte store per half.
template <bool BF16>
__global__ void __launch_bounds__(256) k_pack_b(const float2* __restrict__ x, int Nh, int Nhp, int nrhs, int nel,
                                                const int32_t* __restrict__ elems, const int64_t* __restrict__ off,
                                                int Kp, uint16_t* __restrict__ Bt) {
  auto cvt = [](float f) -> uint32_t {
    if (BF16) {
      const __nv_bfloat16 b = __float2bfloat16_rn(f);
      return *reinterpret_cast<const uint16_t*>(&b);
    }
    const __half h = __float2half_rn(f);
    return *reinterpret_cast<const uint16_t*>(&h);
  };
  const int ng = (Nh + 7) >> 3;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ng * nrhs) return;
  const int g = i / nrhs, c = i - g * nrhs, kb = 8 * g;
  for (int j = blockIdx.y; j < nel; j += gridDim.y) {
    const float2* src = x + (off[elems[j]] + kb) * nrhs + c;
    uint16_t* dre = Bt + ((int64_t)j * nrhs + c) * Kp + kb;
    uint16_t* dim = dre + Nhp;
    if (kb + 8 <= Nh) {
      float2 v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = __ldg(src + (int64_t)t * nrhs);
      uint32_t wr[4], wi[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        wr[t] = cvt(v[2 * t].x) | (cvt(v[2 * t + 1].x) << 16);
        wi[t] = cvt(v[2 * t].y) | (cvt(v[2 * t + 1].y) << 16);
      }
      *reinterpret_cast<uint4*>(dre) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
      *reinterpret_cast<uint4*>(dim) = make_uint4(wi[0], wi[1], wi[2], wi[3]);
    } else {
      for (int t = 0; t < Nh - kb; ++t) {
        const float2 v = __ldg(src + (int64_t)t * nrhs);
        dre[t] = (uint16_t)cvt(v.x);
        dim[t] = (uint16_t)cvt(v.y);
      }
    }
  }
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
std::atomic<int> g_stall_ms{0};
std::once_flag g_encode_once;
int g_sms[64] = {0};

// 2-D tensor map over a row-major (rows x inner) 16-bit matrix with row stride
// ld elements; box = box_inner x box_rows, 128-byte swizzle, zero fill outside.
bool encode_2d(CUtensorMap* m, bool bf16, const void* base, uint64_t inner, uint64_t rows, uint64_t ld,
               uint32_t box_inner, uint32_t box_rows) {
  return tc_encode_2d(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, base, inner,
                      rows, ld * 2, box_inner, box_rows);
}

}  // namespace

bool tc_encode_2d(CUtensorMap* m, CUtensorMapDataType dtype, const void* base, uint64_t inner, uint64_t rows,
                  uint64_t ld_bytes, uint32_t box_inner, uint32_t box_rows) {
  if (!g_encode) return false;
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {ld_bytes};
  const cuuint32_t box[2] = {box_inner, box_rows};
  const cuuint32_t es[2] = {1, 1};
  return g_encode(m, dtype, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int tc_stall_ms() { return g_stall_ms.load(); }

// stage ring + epilogue staging (8 warps x 16 x 17 complex) + alignment slack
size_t tc_smem_bytes() { return (size_t)STAGES * STAGE_BYTES + 8 * 16 * 17 * 8 + 1024; }

int tc_k_split(int Nh) { return (Nh + 7) / 8 * 8; }

// Testing hook (mm_test_tc_stall): a non-zero limit makes the following
// tensor-core kernels issue no products and give up every wait after that many
// milliseconds.
void tc_set_stall(int ms) { g_stall_ms.store(ms < 0 ? 0 : ms); }

cudaError_t tc_gemm_init() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  });
  if (!g_encode) return cudaErrorNotSupported;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64) {
    e = cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes());
  if (e != cudaSuccess) return e;
  return cudaSuccess;
}

namespace {

template <bool BF16>
cudaError_t launch_tc(const CUtensorMap& tmA, const CUtensorMap& tmB, int num_m, int num_n, int nk, int Nh,
                      int ncols, int nrhs, const int32_t* elems, const int64_t* off, float2* u, float2* v, int* err,
                      int sms, cudaStream_t st) {
  const int num_groups = num_m * num_n;
  const int ctas = std::max(1, std::min(sms, num_groups));
  const int stall_ms = g_stall_ms.load();
  const uint64_t wait_ns = stall_ms > 0 ? (uint64_t)stall_ms * 1000000ull : kWaitNs;
  k_tc_gemm<BF16><<<ctas, kThreads, tc_smem_bytes(), st>>>(tmA, tmB, num_m, num_groups, nk, Nh, ncols, nrhs, elems,
                                                          off, u, v, err, wait_ns, stall_ms > 0 ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace

cudaError_t tc_macro_gemm(bool bf16, const uint16_t* A, int Mp, int Kp, int Nh, const int32_t* elems, int nel,
                          int nrhs, const int64_t* off, const float2* x, uint16_t* Bt, size_t bt_cap, float2* u,
                          float2* v, int* err, cudaStream_t st) {
  const int ncols = nel * nrhs;
  if (ncols <= 0) return cudaSuccess;
  const int Nhp = tc_k_split(Nh);
  if (!g_encode || Mp % TBM || Kp % TBK || Nhp + Nh > Kp || (size_t)ncols * Kp > bt_cap) return cudaErrorInvalidValue;
  {
    const int items = ((Nh + 7) / 8) * nrhs;
    dim3 pg((unsigned)((items + 255) / 256), (unsigned)std::min(nel, 65535));
    if (bf16)
      k_pack_b<true><<<pg, 256, 0, st>>>(x, Nh, Nhp, nrhs, nel, elems, off, Kp, Bt);
    else
      k_pack_b<false><<<pg, 256, 0, st>>>(x, Nh, Nhp, nrhs, nel, elems, off, Kp, Bt);
  }
  CUtensorMap tmA, tmB;
  if (!encode_2d(&tmA, bf16, A, (uint64_t)Kp, (uint64_t)Mp, (uint64_t)Kp, TBK, TBM) ||
      !encode_2d(&tmB, bf16, Bt, (uint64_t)(Nhp + Nh), (uint64_t)ncols, (uint64_t)Kp, TBK, TBN))
    return cudaErrorInvalidValue;
  const int num_m = Mp / TBM, num_n = (ncols + TBN - 1) / TBN;
  int dev = 0;
  cudaGetDevice(&dev);
  const int sms = (dev >= 0 && dev < 64 && g_sms[dev] > 0) ? g_sms[dev] : 148;
  const int nk = Kp / TBK;
  return bf16 ? launch_tc<true>(tmA, tmB, num_m, num_n, nk, Nh, ncols, nrhs, elems, off, u, v, err, sms, st)
              : launch_tc<false>(tmA, tmB, num_m, num_n, nk, Nh, ncols, nrhs, elems, off, u, v, err, sms, st);
}

int tc_tile_m() { return TBM; }
int tc_tile_k() { return TBK; }
int tc_tile_n() { return TBN; }

}  // namespace mm
