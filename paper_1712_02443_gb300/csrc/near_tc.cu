// Block near field on tensor cores (Sec. V, the precorrected near-field
// operator G_NF applied as translation-invariant blocks): v -= B_q u_b over all
// element pairs (a, b) coupled by block q, with FP32-level accuracy from TF32
// tensor-core products.
//
// Arithmetic.  Every operand x is split into two TF32 numbers, hi = rn(x) and
// lo = rn(x - hi) (10-bit significands, FP32's exponent range, so no scaling is
// needed); the product is hi_a hi_b + hi_a lo_b + lo_a hi_b with FP32
// accumulation in tensor memory.  The dropped term lo_a lo_b and the rounding
// of lo are each about 2^-22 of |a b|, comparable to FP32 rounding.
//
// Complex product as a real GEMM without expanding the block: block row m is
// the real row [Re B_m0, Im B_m0, Re B_m1, Im B_m1, ...] (the complex block as
// stored, K = 2 Nb real entries), and each complex column u gets two real B
// rows: [Re u_0, -Im u_0, Re u_1, -Im u_1, ...] gives Re(B u) and
// [Im u_0, Re u_0, Im u_1, Re u_1, ...] gives Im(B u).  A tile of NC complex
// columns is an MMA of N = 2 NC: accumulator columns [0, NC) hold the real
// parts, [NC, 2 NC) the imaginary parts.
//
// Work unit: (group g = block q and its element pairs, 128-row tile mt of the
// block, NC-column tile of the group's (pair, right-hand side) columns).  Only
// the 16-complex-column k tiles of (q, mt) that hold a non-zero are visited
// (the block's bases are in anchor order).  Persistent kernel: one CTA per SM
// takes units blockIdx.x, blockIdx.x + gridDim.x, ...; it finds a unit's group
// by a binary search over the per-group prefix of unit counts, built once in
// shared memory.  Roles (448 threads):
//   warp 0     one lane: TMA copies of the A tiles (hi and lo, 128 rows x 32
//              FP32, 128-byte swizzle) into the stage ring;
//   warp 1     allocates two accumulators of 2 NC tensor-memory columns; one
//              lane issues tcgen05.mma kind::tf32 (M 128, N 2 NC, K 8), 12 per
//              k tile, alternating accumulators from unit to unit so that the
//              epilogue of one unit overlaps the products of the next;
//   warps 2-9  gather u for the B tiles: 8-byte cp.async copies of the
//              columns' entries (pair offsets and the column type's anchor
//              order) into a raw ring several k tiles deep, then the split into
//              hi / lo and the two real rows per column, stored swizzled;
//   warps 10-13 epilogue: tensor memory -> registers -> the pair's slice of a
//              partial-sum buffer, P_p[c][m] (consecutive lanes store
//              consecutive rows).
// A row element has one pair per lattice offset, so the slices never overlap
// and need no atomics; k_near_reduce then subtracts the sum of each element's
// slices from v (rows back in basis order).
// Every mbarrier wait is bounded in time; on expiry the kernel sets an error
// flag, the other roles stop, copies and products in flight are waited for
// (bounded) and tensor memory is freed.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "cp_async.cuh"
#include "device.h"
#include "near_tc.h"
#include "tc_gemm.h"
#include "tcgen05.cuh"

namespace mm {

namespace {

using namespace tcx;

constexpr int kRowsT = 128;                 // block rows per tile (MMA M)
constexpr int kKT = 16;                     // complex block columns per k tile (32 FP32 = 128 bytes)
constexpr int kATile = kRowsT * 128;        // bytes of one A tile (hi or lo)
constexpr int kThreadsNT = 448;             // A copies, MMA, 8 gather warps, 4 epilogue warps
constexpr int kProd = 256;                  // gather threads (warps 2-9)
constexpr int kEpi = 128;                   // epilogue threads (warps 10-13)
constexpr int kEpiWarp0 = 2 + kProd / 32;   // first epilogue warp
constexpr int kMaxGroups = 512;             // groups whose unit prefix a CTA keeps in shared memory
constexpr unsigned long long kWaitNs = 1000000000ull;
constexpr unsigned long long kDrainNs = 1000000000ull;

__device__ int g_near_tc_err;               // set when a bounded wait expired

template <int NC, int STAGES, int RAWD>
struct NearTcCfg {
  static constexpr int BTile = 2 * NC * 128;                 // one B tile: 2 NC rows x 32 FP32
  static constexpr int Stage = 2 * kATile + 2 * BTile;       // A hi, A lo, B hi, B lo
  static constexpr int Raw = NC * kKT * 8;                   // one raw k tile: NC columns x 16 complex
  static constexpr size_t Smem = (size_t)STAGES * Stage + (size_t)RAWD * Raw + 1024;
};

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t b = __float_as_uint(x);
  b += 0x0FFFu + ((b >> 13) & 1u);
  return __uint_as_float(b & 0xFFFFE000u);
}

// named barriers of the gather warps (1) and of the epilogue warps (2)
__device__ __forceinline__ void gather_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kProd) : "memory"); }
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 2, %0;" ::"n"(kEpi) : "memory"); }

// D (tensor memory) += A B^T (accumulate = 0 overwrites D), kind::tf32.
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// One work unit: group g (block q, pairs), 128-row tile mt, column tile nt,
// and its non-zero k tiles [e0, e1) of the tile list.
struct Unit {
  int g, q, Na, mt, e0, e1, part;
  int64_t n0, ncol, first_pair;
};

// Unit t from the per-group prefix of unit counts (gpre, shared memory):
// groups in order, then 128-row tiles, then column tiles (fastest).
template <int NC>
__device__ __forceinline__ Unit decode_unit(int64_t tk, const int64_t* gpre, int ngroups,
                                            const NearGroupDev* __restrict__ groups, const int32_t* __restrict__ tptr,
                                            int nmt, int nrhs, int ks) {
  // ks shares of a unit's k tiles are consecutive units
  const int64_t t = tk / ks;
  const int part = (int)(tk - t * ks);
  int lo = 0, hi = ngroups - 1;   // last g with gpre[g] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (gpre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const NearGroupDev gg = groups[lo];
  Unit un;
  un.g = lo;
  un.q = gg.q;
  un.Na = gg.Na;
  un.first_pair = gg.first_pair;
  un.ncol = gg.npairs * nrhs;
  const int64_t nnt = (un.ncol + NC - 1) / NC, r = t - gpre[lo];
  un.mt = (int)(r / nnt);
  un.n0 = (r % nnt) * NC;
  const int ea = tptr[un.q * nmt + un.mt], eb = tptr[un.q * nmt + un.mt + 1];
  un.e0 = ea + (int)((int64_t)(eb - ea) * part / ks);
  un.e1 = ea + (int)((int64_t)(eb - ea) * (part + 1) / ks);
  un.part = part;
  return un;
}

// Direct form: unit t = (row element a, 128-row tile mt, NC right-hand-side
// columns from c0), tiles fastest-varying last; the elements are taken in the
// order aorder (by type, then by index), so that the CTAs working at one time
// read the blocks of one row type (they stay in L2) and the u of a band of
// neighbouring elements.
struct DUnit {
  int a, mt, Na, p0, p1;
  int64_t c0, offa;
  bool live;
};

template <int NC>
__device__ __forceinline__ DUnit decode_dunit(int64_t t, int nmt, int nnt, const int32_t* __restrict__ aorder,
                                              const int32_t* __restrict__ type_of,
                                              const int64_t* __restrict__ tbase, const int32_t* __restrict__ eptr,
                                              const int64_t* __restrict__ off) {
  DUnit un;
  const int64_t per = (int64_t)nmt * nnt;
  const int64_t ai = t / per;
  un.a = aorder[ai];
  const int64_t r = t - ai * per;
  un.mt = (int)(r / nnt);
  un.c0 = (r - (int64_t)un.mt * nnt) * NC;
  const int ta = type_of[un.a];
  un.Na = (int)(tbase[ta + 1] - tbase[ta]);
  un.p0 = eptr[un.a];
  un.p1 = eptr[un.a + 1];
  un.offa = off[un.a];
  un.live = un.mt * kRowsT < un.Na && un.p1 > un.p0;
  return un;
}

// Walks the k tiles of a direct unit: the element's pairs in order (block q,
// column element offset), and for each the non-zero k tiles [tptr, tptr + 1)
// of (q, mt); pairs without one are skipped.
struct KCursor {
  int ip, p1, e, e1, q, mt, nmt;
  int64_t offb;
  const longlong2* qb;
  const int32_t* tptr;
  __device__ __forceinline__ void start(int p0_, int p1_, int mt_, int nmt_, const longlong2* qb_,
                                        const int32_t* tptr_) {
    ip = p0_ - 1;
    p1 = p1_;
    mt = mt_;
    nmt = nmt_;
    qb = qb_;
    tptr = tptr_;
    e = e1 = 0;
    next_pair();
  }
  __device__ __forceinline__ bool valid() const { return ip < p1; }
  __device__ __forceinline__ void next_pair() {
    for (++ip; ip < p1; ++ip) {
      const longlong2 v = qb[ip];
      q = (int)v.x;
      offb = v.y;
      e = tptr[q * nmt + mt];
      e1 = tptr[q * nmt + mt + 1];
      if (e < e1) return;
    }
  }
  __device__ __forceinline__ void advance() {
    if (++e >= e1) next_pair();
  }
};

// number of k tiles of a direct unit
__device__ __forceinline__ int dunit_tiles(const DUnit& un, int nmt, const longlong2* __restrict__ qb,
                                           const int32_t* __restrict__ tptr) {
  int nk = 0;
  if (!un.live) return 0;
  for (int ip = un.p0; ip < un.p1; ++ip) {
    const int q = (int)qb[ip].x;
    nk += tptr[q * nmt + un.mt + 1] - tptr[q * nmt + un.mt];
  }
  return nk;
}

}  // namespace

template <int NC, int STAGES, int RAWD>
__global__ void __launch_bounds__(kThreadsNT, 1) k_near_tc(
    const __grid_constant__ CUtensorMap tmA, int rows_total, const NearGroupDev* __restrict__ groups, int ngroups,
    const longlong2* __restrict__ poff, const int32_t* __restrict__ arow, const int32_t* __restrict__ bnb, int nmt,
    const int32_t* __restrict__ tptr, const int32_t* __restrict__ tlist, const int32_t* __restrict__ perm,
    const int32_t* __restrict__ bpb, const int64_t* __restrict__ prow, int nrhs, int64_t units, int ks,
    int64_t pstride, const float2* __restrict__ u, float2* __restrict__ P, uint64_t wait_ns, int stall) {
  typedef NearTcCfg<NC, STAGES, RAWD> Cfg;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* rawbuf = base + STAGES * Cfg::Stage;
  __shared__ __align__(8) uint64_t full_a[STAGES], full_b[STAGES], empty_bar[STAGES], tfull[2], tempty[2], drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ volatile int s_gok[2], s_eok[2];
  __shared__ int64_t gpre[kMaxGroups + 1];
  __shared__ int64_t cin[NC], cpart[NC];
  volatile int* stop = &abort_flag;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  // ---- per-group prefix of the unit counts (warp 0, 32 groups at a time)
  if (warp == 0) {
    int64_t run = 0;
    for (int g0 = 0; g0 < ngroups; g0 += 32) {
      const int g = g0 + lane;
      int64_t cnt = 0;
      if (g < ngroups) {
        const NearGroupDev gg = groups[g];
        cnt = (int64_t)((gg.Na + kRowsT - 1) / kRowsT) * ((gg.npairs * nrhs + NC - 1) / NC);
      }
      int64_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (g < ngroups) gpre[g] = run + incl - cnt;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
      gpre[ngroups] = run;
      abort_flag = 0;
      for (int s = 0; s < STAGES; ++s) {
        mbar_init(smem_u32(&full_a[s]), 1);
        mbar_init(smem_u32(&full_b[s]), kProd);
        mbar_init(smem_u32(&empty_bar[s]), 1);
      }
      for (int b = 0; b < 2; ++b) {
        mbar_init(smem_u32(&tfull[b]), 1);
        mbar_init(smem_u32(&tempty[b]), kEpi / 32);   // lane 0 of each epilogue warp
      }
      mbar_init(smem_u32(&drain_bar), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)(4 * NC)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- A producer: the hi and lo tiles of every non-zero k tile of every unit
      uint32_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < units && ok; t += gridDim.x) {
        const Unit un = decode_unit<NC>(t, gpre, ngroups, groups, tptr, nmt, nrhs, ks);
        const int row0 = arow[un.q] + un.mt * kRowsT;
        for (int e = un.e0; e < un.e1; ++e, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t r = it / STAGES;
          if (!mbar_wait(smem_u32(&empty_bar[s]), (r & 1) ^ 1, stop, wait_ns)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_a[s]);
          unsigned char* sa = base + s * Cfg::Stage;
          const int x = tlist[e] * 2 * kKT;   // FP32 column of the k tile
          mbar_expect_tx(fb, 2 * kATile);
          tma_load_2d(&tmA, smem_u32(sa), fb, x, row0);
          tma_load_2d(&tmA, smem_u32(sa + kATile), fb, x, row0 + rows_total);
        }
      }
      if (!ok && !*stop) {
        *stop = 1;
        atomicExch(&g_near_tc_err, 1);
      }
      // copies in flight land before the CTA's shared memory is released
      for (uint32_t j = it > (uint32_t)STAGES ? it - STAGES : 0; j < it; ++j)
        mbar_wait(smem_u32(&full_a[j % STAGES]), (j / STAGES) & 1, nullptr, kDrainNs);
    }
  } else if (warp == 1) {
    if (lane == 0 && !stall) {
      // ---- MMA issuer: one accumulator (of two) per unit
      constexpr uint32_t idesc = make_idesc(2u, kRowsT, 2 * NC);
      uint32_t it = 0, lt = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < units && ok; t += gridDim.x) {
        const Unit un = decode_unit<NC>(t, gpre, ngroups, groups, tptr, nmt, nrhs, ks);
        const int nk = un.e1 - un.e0;
        if (nk == 0) continue;
        const uint32_t b = lt & 1, ub = lt >> 1;
        if (!mbar_wait(smem_u32(&tempty[b]), (ub & 1) ^ 1, stop, wait_ns)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + b * (uint32_t)(2 * NC);
        for (int i = 0; i < nk; ++i, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t r = it / STAGES;
          if (!mbar_wait(smem_u32(&full_a[s]), r & 1, stop, wait_ns) ||
              !mbar_wait(smem_u32(&full_b[s]), r & 1, stop, wait_ns)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(base + s * Cfg::Stage);
          const uint64_t dah = make_desc_sw128(sa), dal = make_desc_sw128(sa + kATile);
          const uint64_t dbh = make_desc_sw128(sa + 2 * kATile);
          const uint64_t dbl = make_desc_sw128(sa + 2 * kATile + Cfg::BTile);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {   // K 8 TF32 = 32 bytes per product
            const uint64_t o = (uint64_t)((kk * 32) >> 4);
            mma_tf32(d, dah + o, dbh + o, idesc, (i > 0 || kk > 0) ? 1u : 0u);   // hi a . hi b
            mma_tf32(d, dah + o, dbl + o, idesc, 1u);                            // hi a . lo b
            mma_tf32(d, dal + o, dbh + o, idesc, 1u);                            // lo a . hi b
          }
          umma_commit(smem_u32(&empty_bar[s]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&tfull[b]));
        ++lt;
      }
      if (!ok && !*stop) {
        *stop = 1;
        atomicExch(&g_near_tc_err, 1);
      }
    }
    if (lane == 0) {
      // every product issued here completes before tensor memory and the stages go away
      umma_commit(smem_u32(&drain_bar));
      mbar_wait(smem_u32(&drain_bar), 0, nullptr, kDrainNs);
    }
  } else if (warp < kEpiWarp0) {
    // ---- gather (warps 2-9, pt = 0..255): u of the units' columns -> B tiles
    const int pt = threadIdx.x - 64;
    const uint32_t raw0 = smem_u32(rawbuf);
    uint32_t it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < units && ok; t += gridDim.x) {
      const Unit un = decode_unit<NC>(t, gpre, ngroups, groups, tptr, nmt, nrhs, ks);
      const int nk = un.e1 - un.e0;
      if (nk == 0) continue;   // the same for every gather thread
      gather_sync();           // nobody reads the previous unit's column table any more
      for (int n = pt; n < NC; n += kProd) {
        const int64_t nn = un.n0 + n;
        if (nn < un.ncol) {
          const int64_t pp = nn / nrhs;
          cin[n] = poff[un.first_pair + pp].y * nrhs + (nn - pp * nrhs);   // u index of the column's unknown 0
        } else {
          cin[n] = -1;
        }
      }
      gather_sync();
      const int Nb = bnb[un.q];
      const int32_t* pb = perm + bpb[un.q];
      // raw k tile i -> slot i % RAWD: [column n][16 complex], 8-byte copies;
      // consecutive threads take consecutive columns (consecutive right-hand sides)
      auto issue = [&](int i) {
        if (i < nk) {
          const int kt = tlist[un.e0 + i];
          const uint32_t slot = raw0 + (uint32_t)((i % RAWD) * Cfg::Raw);
#pragma unroll
          for (int r = 0; r < NC * kKT / kProd; ++r) {
            const int h = pt + kProd * r, n = h % NC, kk = h / NC;
            const int k = kt * kKT + kk;
            const int64_t ci = cin[n];
            const bool valid = ci >= 0 && k < Nb;
            const float2* src = valid ? u + ci + (int64_t)__ldg(pb + k) * nrhs : u;
            cp_async8(slot + (uint32_t)(n * kKT + kk) * 8u, src, valid);
          }
        }
        cp_async_commit();
      };
#pragma unroll
      for (int i = 0; i < RAWD - 1; ++i) issue(i);
      for (int i = 0; i < nk; ++i, ++it) {
        const int s = (int)(it % STAGES);
        const uint32_t r = it / STAGES;
        cp_async_wait<RAWD - 2>();   // this thread's copies of k tile i have landed
        // one thread waits for the stage and tells the others through the named
        // barrier, so that all gather threads take the same branch; two flags alternate, so
        // a value is not overwritten before every thread has read it
        if (pt == 0) s_gok[it & 1] = mbar_wait(smem_u32(&empty_bar[s]), (r & 1) ^ 1, stop, wait_ns) ? 1 : 0;
        gather_sync();               // everyone's copies landed; slot (i - 1) % RAWD is free again
        if (!s_gok[it & 1]) {
          ok = false;
          break;
        }
        issue(i + RAWD - 1);
        const uint32_t slot = raw0 + (uint32_t)((i % RAWD) * Cfg::Raw);
        const uint32_t bh = smem_u32(base + s * Cfg::Stage + 2 * kATile), bl = bh + Cfg::BTile;
        // chunk (n, j): complex entries 2j, 2j + 1 of column n (16 bytes of raw);
        // consecutive threads take the 8 chunks of a column (conflict-free)
#pragma unroll
        for (int rr = 0; rr < NC * 8 / kProd; ++rr) {
          const int h = pt + kProd * rr, j = h & 7, n = h >> 3;
          float4 w;
          asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                       : "=f"(w.x), "=f"(w.y), "=f"(w.z), "=f"(w.w)
                       : "r"(slot + (uint32_t)(n * kKT * 8 + j * 16)));
          const float hr0 = tf32_rn(w.x), hi0 = tf32_rn(w.y), hr1 = tf32_rn(w.z), hi1 = tf32_rn(w.w);
          const float lr0 = tf32_rn(w.x - hr0), li0 = tf32_rn(w.y - hi0), lr1 = tf32_rn(w.z - hr1),
                      li1 = tf32_rn(w.w - hi1);
          const uint32_t o1 = (uint32_t)(n * 128 + ((j ^ (n & 7)) << 4));          // row n: real parts
          const uint32_t o2 = (uint32_t)((NC + n) * 128 + ((j ^ (n & 7)) << 4));   // row NC + n: imaginary
          st_shared_v4(bh + o1, hr0, -hi0, hr1, -hi1);
          st_shared_v4(bh + o2, hi0, hr0, hi1, hr1);
          st_shared_v4(bl + o1, lr0, -li0, lr1, -li1);
          st_shared_v4(bl + o2, li0, lr0, li1, lr1);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&full_b[s]));
      }
      cp_async_wait<0>();   // no copy of this unit outlives it
    }
    cp_async_wait<0>();
    if (!ok && !*stop) {
      *stop = 1;
      atomicExch(&g_near_tc_err, 1);
    }
  } else {
    // ---- epilogue (warps 10-13): thread = block row m (TMEM lane), the unit's
    // columns 16 at a time, into the pairs' slices of P
    const int et = threadIdx.x - 32 * kEpiWarp0, qd = warp & 3;
    uint32_t lt = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < units && ok; t += gridDim.x) {
      const Unit un = decode_unit<NC>(t, gpre, ngroups, groups, tptr, nmt, nrhs, ks);
      const int nk = un.e1 - un.e0;
      epi_sync();   // nobody reads the previous unit's column table any more
      for (int n = et; n < NC; n += kEpi) {
        const int64_t nn = un.n0 + n;
        if (nn < un.ncol) {
          const int64_t pp = nn / nrhs;
          cpart[n] = prow[un.first_pair + pp] * nrhs + (nn - pp * nrhs) * un.Na + un.part * pstride;
        } else {
          cpart[n] = -1;
        }
      }
      epi_sync();
      const int m = un.mt * kRowsT + 32 * qd + lane;   // block row (the row type's anchor order)
      if (nk == 0) {
        // no non-zero k tile in these rows: their partial sums are zero
        if (m < un.Na)
          for (int c = 0; c < NC; ++c)
            if (cpart[c] >= 0) P[cpart[c] + m] = make_float2(0.f, 0.f);
        continue;
      }
      const uint32_t b = lt & 1, ub = lt >> 1;
      if (et == 0) s_eok[lt & 1] = mbar_wait(smem_u32(&tfull[b]), ub & 1, stop, wait_ns) ? 1 : 0;
      epi_sync();
      if (!s_eok[lt & 1]) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16) + b * (uint32_t)(2 * NC);
#pragma unroll 1
      for (int c0 = 0; c0 < NC; c0 += 16) {
        uint32_t re[16], im[16];
        tmem_ld16(tl + (uint32_t)c0, re);
        tmem_ld16(tl + (uint32_t)(NC + c0), im);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (m < un.Na) {
#pragma unroll
          for (int c = 0; c < 16; ++c) {   // consecutive lanes: consecutive rows of one column
            const int64_t cp = cpart[c0 + c];
            if (cp >= 0) P[cp + m] = make_float2(__uint_as_float(re[c]), __uint_as_float(im[c]));
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
      ++lt;
    }
    if (!ok && et == 0 && !*stop) {
      *stop = 1;
      atomicExch(&g_near_tc_err, 1);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(4 * NC)));
  }
}

// Direct form of the same products for many right-hand sides: work unit =
// (row element a, 128-row tile mt, NC right-hand-side columns from c0).  Its k
// tiles run over all pairs (a, b) of the element (block q of the pair and its
// non-zero k tiles of row tile mt) into one accumulator, and the epilogue
// subtracts the accumulator from v in place (every (row, column) of v belongs
// to one unit): no partial sums and no reduction pass.  A k tile's B rows are
// 16 basis functions of element b with NC consecutive right-hand sides each,
// copied with 16-byte cp.async (nrhs even, so every row starts 16-byte
// aligned).  Roles, waits and error handling as in k_near_tc.
template <int NC, int STAGES, int RAWD>
__global__ void __launch_bounds__(kThreadsNT, 1) k_near_tc_direct(
    const __grid_constant__ CUtensorMap tmA, int rows_total, const int32_t* __restrict__ arow,
    const int32_t* __restrict__ bnb, int nmt, const int32_t* __restrict__ tptr, const int32_t* __restrict__ tlist,
    const int32_t* __restrict__ perm, const int32_t* __restrict__ bpb, const int32_t* __restrict__ eptr,
    const longlong2* __restrict__ qb, const int32_t* __restrict__ aorder, const int32_t* __restrict__ type_of,
    const int64_t* __restrict__ tbase,
    const int32_t* __restrict__ tperm, const int64_t* __restrict__ off, int nrhs, int64_t units,
    const float2* __restrict__ u, float2* __restrict__ v, uint64_t wait_ns, int stall) {
  typedef NearTcCfg<NC, STAGES, RAWD> Cfg;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* rawbuf = base + STAGES * Cfg::Stage;
  __shared__ __align__(8) uint64_t full_a[STAGES], full_b[STAGES], empty_bar[STAGES], tfull[2], tempty[2], drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ volatile int s_gok[2], s_eok[2];
  volatile int* stop = &abort_flag;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nnt = (nrhs + NC - 1) / NC;

  if (warp == 0 && lane == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_a[s]), 1);
      mbar_init(smem_u32(&full_b[s]), kProd);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), kEpi / 32);
    }
    mbar_init(smem_u32(&drain_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)(4 * NC)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- A producer: hi and lo tiles of every k tile of every pair of the unit
      uint32_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < units && ok; t += gridDim.x) {
        const DUnit un = decode_dunit<NC>(t, nmt, nnt, aorder, type_of, tbase, eptr, off);
        if (!un.live) continue;
        KCursor c;
        for (c.start(un.p0, un.p1, un.mt, nmt, qb, tptr); c.valid(); c.advance(), ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t r = it / STAGES;
          if (!mbar_wait(smem_u32(&empty_bar[s]), (r & 1) ^ 1, stop, wait_ns)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&full_a[s]);
          unsigned char* sa = base + s * Cfg::Stage;
          const int x = tlist[c.e] * 2 * kKT;
          const int row0 = arow[c.q] + un.mt * kRowsT;
          mbar_expect_tx(fb, 2 * kATile);
          tma_load_2d(&tmA, smem_u32(sa), fb, x, row0);
          tma_load_2d(&tmA, smem_u32(sa + kATile), fb, x, row0 + rows_total);
        }
      }
      if (!ok && !*stop) {
        *stop = 1;
        atomicExch(&g_near_tc_err, 1);
      }
      for (uint32_t j = it > (uint32_t)STAGES ? it - STAGES : 0; j < it; ++j)
        mbar_wait(smem_u32(&full_a[j % STAGES]), (j / STAGES) & 1, nullptr, kDrainNs);
    }
  } else if (warp == 1) {
    if (lane == 0 && !stall) {
      // ---- MMA issuer: one accumulator (of two) per unit, over all its k tiles
      constexpr uint32_t idesc = make_idesc(2u, kRowsT, 2 * NC);
      uint32_t it = 0, lt = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < units && ok; t += gridDim.x) {
        const DUnit un = decode_dunit<NC>(t, nmt, nnt, aorder, type_of, tbase, eptr, off);
        const int nk = dunit_tiles(un, nmt, qb, tptr);
        if (nk == 0) continue;
        const uint32_t b = lt & 1, ub = lt >> 1;
        if (!mbar_wait(smem_u32(&tempty[b]), (ub & 1) ^ 1, stop, wait_ns)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + b * (uint32_t)(2 * NC);
        for (int i = 0; i < nk; ++i, ++it) {
          const int s = (int)(it % STAGES);
          const uint32_t r = it / STAGES;
          if (!mbar_wait(smem_u32(&full_a[s]), r & 1, stop, wait_ns) ||
              !mbar_wait(smem_u32(&full_b[s]), r & 1, stop, wait_ns)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(base + s * Cfg::Stage);
          const uint64_t dah = make_desc_sw128(sa), dal = make_desc_sw128(sa + kATile);
          const uint64_t dbh = make_desc_sw128(sa + 2 * kATile);
          const uint64_t dbl = make_desc_sw128(sa + 2 * kATile + Cfg::BTile);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t o = (uint64_t)((kk * 32) >> 4);
            mma_tf32(d, dah + o, dbh + o, idesc, (i > 0 || kk > 0) ? 1u : 0u);
            mma_tf32(d, dah + o, dbl + o, idesc, 1u);
            mma_tf32(d, dal + o, dbh + o, idesc, 1u);
          }
          umma_commit(smem_u32(&empty_bar[s]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&tfull[b]));
        ++lt;
      }
      if (!ok && !*stop) {
        *stop = 1;
        atomicExch(&g_near_tc_err, 1);
      }
    }
    if (lane == 0) {
      umma_commit(smem_u32(&drain_bar));
      mbar_wait(smem_u32(&drain_bar), 0, nullptr, kDrainNs);
    }
  } else if (warp < kEpiWarp0) {
    // ---- gather (warps 2-9, pt = 0..255): rows of u -> B tiles
    const int pt = threadIdx.x - 64;
    const uint32_t raw0 = smem_u32(rawbuf);
    uint32_t it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < units && ok; t += gridDim.x) {
      const DUnit un = decode_dunit<NC>(t, nmt, nnt, aorder, type_of, tbase, eptr, off);
      const int nk = dunit_tiles(un, nmt, qb, tptr);
      if (nk == 0) continue;   // the same for every gather thread
      KCursor pre;
      pre.start(un.p0, un.p1, un.mt, nmt, qb, tptr);
      // raw k tile i -> slot i % RAWD: [k row kk][column n], 16-byte copies of two
      // right-hand sides; consecutive threads take consecutive pieces of a row
      auto issue = [&](int i) {
        if (i < nk) {
          const int kt = tlist[pre.e];
          const int Nb = bnb[pre.q];
          const int32_t* pb = perm + bpb[pre.q];
          const int64_t ob = pre.offb;
          const uint32_t slot = raw0 + (uint32_t)((i % RAWD) * Cfg::Raw);
#pragma unroll
          for (int r = 0; r < NC * kKT / 2 / kProd; ++r) {
            const int h = pt + kProd * r, kk = h / (NC / 2), m2 = h - kk * (NC / 2);
            const int k = kt * kKT + kk;
            const int64_t c = un.c0 + 2 * m2;
            const bool valid = k < Nb && c < nrhs;
            const float2* src = valid ? u + ((ob + (int64_t)__ldg(pb + k)) * nrhs + c) : u;
            cp_async16(slot + (uint32_t)(kk * NC + 2 * m2) * 8u, src, valid ? 16u : 0u);
          }
          pre.advance();
        }
        cp_async_commit();
      };
#pragma unroll
      for (int i = 0; i < RAWD - 1; ++i) issue(i);
      for (int i = 0; i < nk; ++i, ++it) {
        const int s = (int)(it % STAGES);
        const uint32_t r = it / STAGES;
        cp_async_wait<RAWD - 2>();
        if (pt == 0) s_gok[it & 1] = mbar_wait(smem_u32(&empty_bar[s]), (r & 1) ^ 1, stop, wait_ns) ? 1 : 0;
        gather_sync();
        if (!s_gok[it & 1]) {
          ok = false;
          break;
        }
        issue(i + RAWD - 1);
        const uint32_t slot = raw0 + (uint32_t)((i % RAWD) * Cfg::Raw);
        const uint32_t bh = smem_u32(base + s * Cfg::Stage + 2 * kATile), bl = bh + Cfg::BTile;
        // chunk (n, j): complex entries 2j, 2j + 1 of column n; consecutive
        // threads take consecutive columns (conflict-free reads of the raw rows,
        // and the swizzle spreads the 16-byte stores over all banks)
#pragma unroll
        for (int rr = 0; rr < NC * 8 / kProd; ++rr) {
          const int h = pt + kProd * rr, n = h % NC, j = h / NC;
          float2 e0, e1;
          asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(e0.x), "=f"(e0.y)
                       : "r"(slot + (uint32_t)((2 * j) * NC + n) * 8u));
          asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(e1.x), "=f"(e1.y)
                       : "r"(slot + (uint32_t)((2 * j + 1) * NC + n) * 8u));
          const float hr0 = tf32_rn(e0.x), hi0 = tf32_rn(e0.y), hr1 = tf32_rn(e1.x), hi1 = tf32_rn(e1.y);
          const float lr0 = tf32_rn(e0.x - hr0), li0 = tf32_rn(e0.y - hi0), lr1 = tf32_rn(e1.x - hr1),
                      li1 = tf32_rn(e1.y - hi1);
          const uint32_t o1 = (uint32_t)(n * 128 + ((j ^ (n & 7)) << 4));
          const uint32_t o2 = (uint32_t)((NC + n) * 128 + ((j ^ (n & 7)) << 4));
          st_shared_v4(bh + o1, hr0, -hi0, hr1, -hi1);
          st_shared_v4(bh + o2, hi0, hr0, hi1, hr1);
          st_shared_v4(bl + o1, lr0, -li0, lr1, -li1);
          st_shared_v4(bl + o2, li0, lr0, li1, lr1);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_u32(&full_b[s]));
      }
      cp_async_wait<0>();
    }
    cp_async_wait<0>();
    if (!ok && !*stop) {
      *stop = 1;
      atomicExch(&g_near_tc_err, 1);
    }
  } else {
    // ---- epilogue (warps 10-13): thread = block row m (TMEM lane); v row of
    // the row element (anchor order -> basis), 16 columns at a time, v -= acc
    const int et = threadIdx.x - 32 * kEpiWarp0, qd = warp & 3;
    uint32_t lt = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < units && ok; t += gridDim.x) {
      const DUnit un = decode_dunit<NC>(t, nmt, nnt, aorder, type_of, tbase, eptr, off);
      const int nk = dunit_tiles(un, nmt, qb, tptr);
      if (nk == 0) continue;
      const int m = un.mt * kRowsT + 32 * qd + lane;
      const uint32_t b = lt & 1, ub = lt >> 1;
      if (et == 0) s_eok[lt & 1] = mbar_wait(smem_u32(&tfull[b]), ub & 1, stop, wait_ns) ? 1 : 0;
      epi_sync();
      if (!s_eok[lt & 1]) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16) + b * (uint32_t)(2 * NC);
      float2* row = nullptr;
      if (m < un.Na) {
        const int32_t* pa = perm + tperm[type_of[un.a]];
        row = v + (un.offa + pa[m]) * nrhs + un.c0;
      }
#pragma unroll 1
      for (int c0 = 0; c0 < NC; c0 += 16) {
        uint32_t re[16], im[16];
        tmem_ld16(tl + (uint32_t)c0, re);
        tmem_ld16(tl + (uint32_t)(NC + c0), im);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row != nullptr) {
#pragma unroll
          for (int c = 0; c < 16; c += 2) {   // two right-hand sides per 16-byte access (nrhs even)
            if (un.c0 + c0 + c < nrhs) {
              float4* d = reinterpret_cast<float4*>(row + c0 + c);
              float4 o = *d;
              o.x -= __uint_as_float(re[c]);
              o.y -= __uint_as_float(im[c]);
              o.z -= __uint_as_float(re[c + 1]);
              o.w -= __uint_as_float(im[c + 1]);
              *d = o;
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
      ++lt;
    }
    if (!ok && et == 0 && !*stop) {
      *stop = 1;
      atomicExch(&g_near_tc_err, 1);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(4 * NC)));
  }
}

namespace {

template <int NC, int STAGES, int RAWD>
cudaError_t near_tc_launch_t(const DevArray& a, const DevPrec<float>& p, int nrhs, const float2* u, float2* P,
                             int ks, cudaStream_t st) {
  int64_t units = 0;
  for (const auto& g : a.nfg)
    units += (int64_t)((g.Na + kRowsT - 1) / kRowsT) * ((g.npairs * nrhs + NC - 1) / NC);
  units *= ks;
  if (units == 0) return cudaSuccess;
  if ((int64_t)a.nfg.size() > kMaxGroups) return cudaErrorInvalidValue;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ctas = (int)std::min<int64_t>(units, std::max(1, sms));
  const int stall_ms = tc_stall_ms();
  const uint64_t wait_ns = stall_ms > 0 ? (uint64_t)stall_ms * 1000000ull : kWaitNs;
  typedef NearTcCfg<NC, STAGES, RAWD> Cfg;
  k_near_tc<NC, STAGES, RAWD><<<ctas, kThreadsNT, Cfg::Smem, st>>>(
      p.nfb_tmap, a.nfb_tc_rows, reinterpret_cast<const NearGroupDev*>(a.nfg_dev), (int)a.nfg.size(), a.nfg_poff,
      a.nfb_arow, a.nfb_nb, a.nfb_nmt128, a.nfb_tptr128, a.nfb_tlist128, a.nfb_perm, a.nfb_pb, a.nfg_prow, nrhs,
      units, ks, a.nfg_prows * (int64_t)nrhs, u, P, wait_ns, stall_ms > 0 ? 1 : 0);
  return cudaGetLastError();
}

template <int NC, int STAGES, int RAWD>
cudaError_t near_tc_direct_launch_t(const DevArray& a, const DevPrec<float>& p, int nrhs, const float2* u, float2* v,
                                    cudaStream_t st) {
  if (nrhs % 2 != 0 || (reinterpret_cast<uintptr_t>(u) & 15) != 0 || (reinterpret_cast<uintptr_t>(v) & 15) != 0 ||
      a.nfe_qb == nullptr || a.nfe_order == nullptr)
    return cudaErrorInvalidValue;
  const int64_t nnt = (nrhs + NC - 1) / NC;
  const int64_t units = a.n_elem * (int64_t)a.nfb_nmt128 * nnt;
  if (units == 0) return cudaSuccess;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ctas = (int)std::min<int64_t>(units, std::max(1, sms));
  const int stall_ms = tc_stall_ms();
  const uint64_t wait_ns = stall_ms > 0 ? (uint64_t)stall_ms * 1000000ull : kWaitNs;
  typedef NearTcCfg<NC, STAGES, RAWD> Cfg;
  k_near_tc_direct<NC, STAGES, RAWD><<<ctas, kThreadsNT, Cfg::Smem, st>>>(
      p.nfb_tmap, a.nfb_tc_rows, a.nfb_arow, a.nfb_nb, a.nfb_nmt128, a.nfb_tptr128, a.nfb_tlist128, a.nfb_perm,
      a.nfb_pb, a.nfe_ptr, a.nfe_qb, a.nfe_order, a.type_of, a.tbase, a.nfb_tperm, a.off, nrhs, units, u, v, wait_ns,
      stall_ms > 0 ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace

cudaError_t near_tc_init(DevArray& a) {
  cudaError_t e = cudaFuncSetAttribute(k_near_tc<32, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)NearTcCfg<32, 4, 4>::Smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_near_tc<64, 3, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)NearTcCfg<64, 3, 3>::Smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_near_tc_direct<32, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)NearTcCfg<32, 4, 4>::Smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_near_tc_direct<64, 3, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)NearTcCfg<64, 3, 3>::Smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_near_tc_direct<64, 2, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)NearTcCfg<64, 2, 3>::Smem);
  if (e != cudaSuccess) return e;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_near_tc_err);
  if (e != cudaSuccess) return e;
  a.near_err = static_cast<int*>(p);
  return cudaSuccess;
}

// v[a, pa[m]] -= sum over the pairs p of row element a of P_p[c][m] (pa: the
// row type's anchor order -> basis).  One CTA per element; with several
// right-hand sides, 32-row x 32-column chunks pass through shared memory so
// that the partial sums (rows fastest) and v (right-hand sides fastest) are
// both read and written with consecutive threads on consecutive addresses.
__global__ void __launch_bounds__(256) k_near_reduce(const int32_t* __restrict__ eptr,
                                                     const int32_t* __restrict__ epair,
                                                     const int64_t* __restrict__ prow,
                                                     const int32_t* __restrict__ type_of,
                                                     const int64_t* __restrict__ tbase,
                                                     const int32_t* __restrict__ tperm,
                                                     const int32_t* __restrict__ perm, const int64_t* __restrict__ off,
                                                     int nrhs, int ks, int64_t pstride, const float2* __restrict__ P,
                                                     float2* __restrict__ v) {
  constexpr int kMaxPairs = 64;
  __shared__ int64_t sp[kMaxPairs];
  __shared__ float2 tile[32][33];
  const int a = blockIdx.x;
  const int p0 = eptr[a], np = eptr[a + 1] - p0;
  if (np == 0) return;
  const int t = type_of[a];
  const int Na = (int)(tbase[t + 1] - tbase[t]);
  const int32_t* pa = perm + tperm[t];
  const int64_t va = off[a] * nrhs;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (int i = tid; i < np && i < kMaxPairs; i += blockDim.x) sp[i] = prow[epair[p0 + i]] * nrhs;
  __syncthreads();
  auto base = [&](int i) -> int64_t { return i < kMaxPairs ? sp[i] : prow[epair[p0 + i]] * nrhs; };
  if (nrhs == 1) {
    for (int m = tid; m < Na; m += blockDim.x) {
      float2 acc = make_float2(0.f, 0.f);
      for (int i = 0; i < np; ++i)
        for (int h = 0; h < ks; ++h) {
          const float2 x = P[base(i) + h * pstride + m];
          acc.x += x.x;
          acc.y += x.y;
        }
      float2* d = v + va + pa[m];
      float2 o = *d;
      o.x -= acc.x;
      o.y -= acc.y;
      *d = o;
    }
    return;
  }
  for (int m0 = 0; m0 < Na; m0 += 32)
    for (int c0 = 0; c0 < nrhs; c0 += 32) {
      const int m = m0 + lane;
      for (int cc = w; cc < 32; cc += 8) {
        const int c = c0 + cc;
        float2 acc = make_float2(0.f, 0.f);
        if (m < Na && c < nrhs)
          for (int i = 0; i < np; ++i)
            for (int h = 0; h < ks; ++h) {
              const float2 x = P[base(i) + h * pstride + (int64_t)c * Na + m];
              acc.x += x.x;
              acc.y += x.y;
            }
        tile[lane][cc] = acc;
      }
      __syncthreads();
      const int c = c0 + lane;
      for (int mm = w; mm < 32; mm += 8) {
        const int mr = m0 + mm;
        if (mr < Na && c < nrhs) {
          float2* d = v + va + (int64_t)pa[mr] * nrhs + c;
          float2 o = *d;
          o.x -= tile[mm][lane].x;
          o.y -= tile[mm][lane].y;
          *d = o;
        }
      }
      __syncthreads();
    }
}

bool near_tc_direct_ok(const DevArray& a, int nrhs, const void* u, const void* v) {
  return nrhs % 2 == 0 && a.nfe_qb != nullptr && a.nfe_order != nullptr && (reinterpret_cast<uintptr_t>(u) & 15) == 0 &&
         (reinterpret_cast<uintptr_t>(v) & 15) == 0;
}

cudaError_t near_tc_launch(int shape, const DevArray& a, const DevPrec<float>& p, int nrhs, const float2* u,
                           float2* v, float2* P, int ks, cudaStream_t st) {
  if (!p.nfb_tc || a.nfb_tptr128 == nullptr || a.nfe_ptr == nullptr) return cudaErrorInvalidValue;
  if (shape >= 2)
    return shape == 4   ? near_tc_direct_launch_t<64, 2, 3>(a, p, nrhs, u, v, st)
           : shape == 3 ? near_tc_direct_launch_t<64, 3, 3>(a, p, nrhs, u, v, st)
                        : near_tc_direct_launch_t<32, 4, 4>(a, p, nrhs, u, v, st);
  if (P == nullptr) return cudaErrorInvalidValue;
  ks = ks == 2 ? 2 : 1;
  cudaError_t e = shape == 1 ? near_tc_launch_t<64, 3, 3>(a, p, nrhs, u, P, ks, st)
                             : near_tc_launch_t<32, 4, 4>(a, p, nrhs, u, P, ks, st);
  if (e != cudaSuccess) return e;
  k_near_reduce<<<(unsigned)a.n_elem, 256, 0, st>>>(a.nfe_ptr, a.nfe_pair, a.nfg_prow, a.type_of, a.tbase,
                                                    a.nfb_tperm, a.nfb_perm, a.off, nrhs, ks,
                                                    a.nfg_prows * (int64_t)nrhs, P, v);
  return cudaGetLastError();
}

// Host split of the blocks into TF32 hi / lo, same rounding as the kernel's
// (round to nearest even at 10 significand bits); lo is rounded from the
// exact difference (computed in FP64).
static float tf32_rn_host(double v) {
  float f = (float)v;
  uint32_t b;
  std::memcpy(&b, &f, 4);
  b += 0x0FFFu + ((b >> 13) & 1u);
  b &= 0xFFFFE000u;
  std::memcpy(&f, &b, 4);
  return f;
}

void near_tc_split(double re, double im, float* hi, float* lo) {
  hi[0] = tf32_rn_host(re);
  hi[1] = tf32_rn_host(im);
  lo[0] = tf32_rn_host(re - (double)hi[0]);
  lo[1] = tf32_rn_host(im - (double)hi[1]);
}

}  // namespace mm
