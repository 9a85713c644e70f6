// Persistent split-precision stripe GEMM on tcgen05 (sm_103a).
//
// Operands are pre-tiled "slabs": an R x K FP64 matrix (R = M or N side,
// K-major) cut into S BF16 slices, stored as 128-row x 16-K sub-tiles of
// 4 KB in the UMMA no-swizzle K-major core-matrix layout (core matrix
// (mi, ki) at (mi*2 + ki)*128 bytes, row r%8 at 16*(r%8)); for each
// (row tile, K stage) the S slices follow each other (S*4 KB, one bulk
// copy).  Slice i holds q_i * 2^-8i where q_i are the integers peeled from
// x * 2^(8 - sigma_row) (|x| < 2^sigma_row): |q_0| <= 256, |q_i| <= 128.
//
// One job = one 128 x 128 output tile and a list of items (A slab, B slab,
// K stages); all items of a job share the row and column scales, so the
// K-concatenated stripe sum_items A_item . B_item^T accumulates in TMEM
// without a separate reduction (the stripe product of Sec. III.A).  Slice
// pairs (i, j), i + j < S, go to four FP32 TMEM accumulators (512 columns)
// by level l = min(i + j, 3).  Levels 0, 1 and 2 hold integer multiples of
// their unit 2^-8l below 2^24 for K chunks of 192 (level 2 grows by at most
// 2*256*128 + 128^2 = 2^16.3 per K, 192 K give 2^23.9), hence are exact whatever
// rounding the tensor core applies when it adds into the accumulator
// (it truncates: a shared tail accumulator of many pairs would collect a
// biased error of order #adds * 2^-23 of its size); level 3 carries the
// 2^-24-weighted tail.  A chunk is up to 192 K of one item; after it the
// drain warps fold the four levels into a float-float register accumulator
// (K2: scaled by the item's per-column factor, so every task keeps its own
// S*8 bits); the first MMA of the next chunk into each level overwrites it.
// At the end of the job they write the tile (K1: float-float T; K2: F += FP64).
//
// Warp roles (576 threads): warp 0 bulk-copy producer and job fetcher
// (dynamic schedule: an atomic job counter, handed to the other roles through
// a shared-memory ring), warp 1 MMA issuer, warps 2..17 drain/epilogue (TMEM
// lane quarter w%4, 32-column group (w-2)/4).
// Every mbarrier wait is bounded; on timeout the CTA records a status,
// stops issuing, waits (bounded) for its own copies and MMAs, frees TMEM and
// returns.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace su2 {
namespace sp {

constexpr int kRows = 128;           // M tile = N tile
constexpr int kKS = 16;              // K per pipeline stage (one MMA K step)
constexpr int kSub = kRows * kKS * 2;  // bytes of one 128 x 16 BF16 sub-tile
constexpr int kMaxS = 6;
constexpr int kStages = 4;
constexpr int kLead = 8;             // leading slice |q_0| <= 2^kLead, the others |q_i| <= 128
constexpr int kChunkStages = 12;     // 192 K per exact drain
constexpr int kRing = 4;             // job ring slots
constexpr int kThreads = 576;      // producer + MMA + 16 drain warps
constexpr long kSpinLimit = 1L << 26;

struct Item {
  int64_t a_off, b_off;  // byte offsets of the first (row tile, K stage) group
  int32_t nst;           // K stages of 16
  int32_t pad;
  int64_t sc_off;        // MODE_F: offset of the item's per-column drain exponents (a multiple of 128), -1 otherwise
};
// MODE_F: task t's B slab is cut relative to its own column exponents; the
// drain multiplies each chunk of t by 2^d, d = dexp[sc_off + col] =
// own(col) - gamma(col) in [-126, 0], or -127 for a column that is zero (an
// exact power of two, <= 1) before adding it to the tile accumulator.  The
// per-task vector is padded to whole 128-column tiles.
struct TaskScale {
  const int8_t* dexp;
};
struct Job {
  int64_t out_off;       // element offset of the output block
  int32_t rows, cols;    // valid extent of the output block
  int32_t ld, tr, tc;    // leading dimension (rows of the block), tile indices
  int32_t i0, i1;        // items
  int32_t rsc, csc;      // offsets of the row / column exponent arrays
  int32_t nst;           // total K stages of all items
  int32_t nmma;          // MMA N of this tile: the valid columns rounded up to 16 (<= 128)
  int32_t pad2;
};

enum { MODE_T = 0, MODE_F = 1 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; false on timeout or when another role aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (long it = 0; it < kSpinLimit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  return false;
}

// bounded wait by every lane of a warp, then a warp vote: the warp leaves
// converged (the .sync.aligned TMEM loads that follow need that) and agrees
// on success
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  const bool got = mbar_wait(bar, parity, abort_flag);
  return __all_sync(0xffffffffu, got);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  // no swizzle, K-major: LBO = 128 B (next core matrix along K), SBO = 256 B
  // (next 8-row group), descriptor version 1 (bit 46)
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(256 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::f16, A = B = BF16, D = F32, both K-major, M = 128, N = n (multiple of 16)
__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t(n) >> 3) << 17) | ((128u >> 4) << 24);
}

// D (+)= A * B^T; ACC = false overwrites D
template <bool ACC>
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc) {
  if (ACC)
    asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;" ::"r"(tmem), "l"(a), "l"(b), "r"(idesc));
  else
    asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 0;" ::"r"(tmem), "l"(a), "l"(b), "r"(idesc));
}

// the S(S+1)/2 slice products of one 16-K stage, unrolled: pair (i, j) goes to
// level min(i + j, 3); da / db describe slice 0 of A / B, slice i sits kSub
// bytes further (the descriptor's address field counts 16-byte units).  In the
// first stage of a chunk the first product into each level, (0, level),
// overwrites it.
template <int S, bool FIRST>
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc) {
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int jj = 0; jj < S - i; ++jj) {
      const int lvl = (i + jj) < 3 ? (i + jj) : 3;
      const uint64_t a = da + (uint64_t)(i * (kSub >> 4));
      const uint64_t b = db + (uint64_t)(jj * (kSub >> 4));
      if (FIRST && i == 0 && jj == lvl) mma_bf16<false>(tmem + lvl * kRows, a, b, idesc);
      else mma_bf16<true>(tmem + lvl * kRows, a, b, idesc);
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// four 32x32b.x4 TMEM loads (one per accumulator level) and the wait in one
// asm statement: tcgen05.ld writes its destination registers asynchronously,
// so they must not exist as values in the program before tcgen05.wait::ld
// (a separate wait statement would let the compiler reuse or read them early)
__device__ __forceinline__ void tmem_ld4x4_wait(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                                float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%16];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%17];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8,%9,%10,%11}, [%18];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12,%13,%14,%15}, [%19];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_zero8(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr), "r"(z)
               : "memory");
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// x * 2^k for float, exact while the result stays normal
__device__ __forceinline__ float ldexp_f(float x, int k) { return ldexpf(x, k); }

template <int MODE, int S>
__global__ void __launch_bounds__(kThreads, 1)
    split_gemm_kernel(const Job* __restrict__ jobs, int njobs, const Item* __restrict__ items,
                      const unsigned char* __restrict__ Aslab, const unsigned char* __restrict__ Bslab,
                      const int* __restrict__ rexp, const int* __restrict__ cexp, int shift,
                      float* __restrict__ Th, float* __restrict__ Tl, double* __restrict__ F, int* __restrict__ status,
                      int* __restrict__ job_counter, TaskScale ts) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int stage_bytes = 2 * S * kSub;
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], accf_bar, acce_bar, done_bar;
  __shared__ __align__(8) uint64_t jq_full[kRing], jq_empty[kRing];
  __shared__ int job_ring[kRing];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ int issued[kStages];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[s])));
      issued[s] = 0;
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf_bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 512;" ::"r"(smem_u32(&acce_bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done_bar)));
    for (int r = 0; r < kRing; ++r) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&jq_full[r])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 513;" ::"r"(smem_u32(&jq_empty[r])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const int nlev = S < 4 ? S : 4;
  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int st = 0;
      uint32_t use[kStages] = {0, 0, 0, 0};
      bool ok = true;
      for (int k = 0; ok; ++k) {
        const int slot = k % kRing;
        if (!mbar_wait(smem_u32(&jq_empty[slot]), ((k / kRing) & 1) ^ 1, &abort_flag)) {
          ok = false;
          break;
        }
        const int jnext = atomicAdd(job_counter, 1);
        const int j = jnext < njobs ? jnext : -1;
        job_ring[slot] = j;
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&jq_full[slot])) : "memory");
        if (j < 0) break;
        const Job jb = jobs[j];
        const int bbytes = jb.nmma * 32;  // first nmma rows of each B slice sub-tile
        const int tx = S * kSub + S * bbytes;
        for (int it = jb.i0; it < jb.i1 && ok; ++it) {
          const Item item = items[it];
          for (int ks = 0; ks < item.nst; ++ks) {
            if (!mbar_wait(smem_u32(&empty_bar[st]), (use[st] & 1) ^ 1, &abort_flag)) {
              ok = false;
              break;
            }
            const uint32_t fb = smem_u32(&full_bar[st]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(tx) : "memory");
            const uint32_t dst = smem_u32(smem + st * stage_bytes);
            const unsigned char* srcA = Aslab + item.a_off + (int64_t)ks * S * kSub;
            const unsigned char* srcB = Bslab + item.b_off + (int64_t)ks * S * kSub;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                "l"(srcA), "r"(S * kSub), "r"(fb)
                : "memory");
            for (int jj = 0; jj < S; ++jj)
              asm volatile(
                  "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                      dst + S * kSub + jj * kSub),
                  "l"(srcB + jj * kSub), "r"(bbytes), "r"(fb)
                  : "memory");
            issued[st] = (int)use[st] + 1;
            use[st] += 1;
            st = (st + 1) % kStages;
          }
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(status, 4);
      }
      // wait (bounded) for every copy this CTA issued
      for (int s = 0; s < kStages; ++s)
        if (issued[s] > 0) {
          bool fin = false;
          for (long it = 0; it < kSpinLimit && !fin; ++it) fin = mbar_try(smem_u32(&full_bar[s]), (issued[s] - 1) & 1);
          if (!fin) atomicExch(status, 4);
        }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int st = 0;
      uint32_t use[kStages] = {0, 0, 0, 0};
      uint32_t chunk = 0;
      bool ok = true;
      for (int k = 0; ok; ++k) {
        const int slot = k % kRing;
        if (!mbar_wait(smem_u32(&jq_full[slot]), (k / kRing) & 1, &abort_flag)) {
          ok = false;
          break;
        }
        const int j = job_ring[slot];
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&jq_empty[slot])) : "memory");
        if (j < 0) break;
        const Job jb = jobs[j];
        const uint32_t idesc = idesc_n(jb.nmma);
        for (int it = jb.i0; it < jb.i1 && ok; ++it) {
          const int nst = items[it].nst;
          for (int ks = 0; ks < nst; ++ks) {
            const int cpos = ks % kChunkStages;  // a chunk = up to kChunkStages stages of one item
            if (cpos == 0) {
              if (!mbar_wait(smem_u32(&acce_bar), (chunk & 1) ^ 1, &abort_flag)) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;");
            }
            if (!mbar_wait(smem_u32(&full_bar[st]), use[st] & 1, &abort_flag)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = smem_u32(smem + st * stage_bytes);
            const uint64_t da = make_desc(sa), db = make_desc(sa + S * kSub);
            if (cpos == 0) issue_stage<S, true>(tmem, da, db, idesc);
            else issue_stage<S, false>(tmem, da, db, idesc);
            mma_commit(smem_u32(&empty_bar[st]));
            use[st] += 1;
            st = (st + 1) % kStages;
            if (cpos == kChunkStages - 1 || ks == nst - 1) {
              mma_commit(smem_u32(&accf_bar));
              chunk += 1;
            }
          }
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(status, 4);
      }
      // all MMAs issued by this thread complete before TMEM is released
      mma_commit(smem_u32(&done_bar));
      bool fin = false;
      for (long it = 0; it < kSpinLimit && !fin; ++it) fin = mbar_try(smem_u32(&done_bar), 0);
      if (!fin) atomicExch(status, 4);
    }
  } else {
    // ------------------------------------------------------------ drain / epilogue
    const int q = warp & 3;             // TMEM lane quarter
    const int cgrp = (warp - 2) >> 2;   // 32-column group
    const int row = q * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
    uint32_t chunk = 0;
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int slot = k % kRing;
      if (!warp_wait(smem_u32(&jq_full[slot]), (k / kRing) & 1, &abort_flag)) {
        ok = false;
        break;
      }
      const int j = job_ring[slot];
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&jq_empty[slot])) : "memory");
      if (j < 0) break;
      const Job jb = jobs[j];
      float hi[32], lo[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        hi[c] = 0.f;
        lo[c] = 0.f;
      }
      const int ncg4 = min(8, max(0, (jb.nmma - cgrp * 32 + 3) / 4));
      const int c0 = jb.tc * kRows + cgrp * 32;
      for (int it = jb.i0; it < jb.i1 && ok; ++it) {
        const Item item = items[it];
        // MODE_F: this thread's 32 drain exponents of the item, fetched before
        // the chunk wait (two 16-byte loads; byte k of word w = column 4w + k)
        uint32_t dx[8];
        if (MODE == MODE_F) {
          const int4* p = reinterpret_cast<const int4*>(ts.dexp + item.sc_off + c0);
          const int4 u0 = __ldg(p), u1 = __ldg(p + 1);
          dx[0] = u0.x, dx[1] = u0.y, dx[2] = u0.z, dx[3] = u0.w;
          dx[4] = u1.x, dx[5] = u1.y, dx[6] = u1.z, dx[7] = u1.w;
        }
        const int nch = (item.nst + kChunkStages - 1) / kChunkStages;
        for (int ch = 0; ch < nch; ++ch) {
          if (!warp_wait(smem_u32(&accf_bar), chunk & 1, &abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
          for (int cg = 0; cg < 8; ++cg) {
            if (cg >= ncg4) break;
            const uint32_t col = cgrp * 32 + cg * 4;
            float xx[16];  // levels 0..3, four columns each
            tmem_ld4x4_wait(lane_addr + col, lane_addr + 128 + col, lane_addr + 256 + col, lane_addr + 384 + col,
                            xx);
            float x0[4], x1[4], x2[4], x3[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              x0[c] = xx[c];
              x1[c] = xx[4 + c];
              x2[c] = xx[8 + c];
              x3[c] = xx[12 + c];
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const float y1 = nlev > 1 ? x1[c] : 0.f;
              const float y2 = nlev > 2 ? x2[c] : 0.f;
              const float y3 = nlev > 3 ? x3[c] : 0.f;
              float f = 1.f;
              if (MODE == MODE_F) {
                const int d = (int)(int8_t)(dx[cg] >> (8 * c));
                f = __int_as_float((127 + d) << 23);  // 2^d; d = -127 gives 0
              }
              float s, e, h, e2;
              two_sum(x0[c] * f, y1 * f, s, e);
              two_sum(hi[cg * 4 + c], s, h, e2);
              const float l = lo[cg * 4 + c] + (e2 + (e + (y2 * f + y3 * f)));
              const float hs = h + l;
              lo[cg * 4 + c] = l - (hs - h);
              hi[cg * 4 + c] = hs;
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;");
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar)) : "memory");
          chunk += 1;
        }
      }
      if (!ok) break;
      // epilogue: scale by 2^(rexp + cexp - shift) and write
      const int r = jb.tr * kRows + row;
      if (r < jb.rows) {
        const int er = rexp[jb.rsc + r];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          int ce[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) ce[c] = (c0 + g * 8 + c < jb.cols) ? cexp[jb.csc + c0 + g * 8 + c] : 0;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int cc = c0 + g * 8 + c;
            if (cc < jb.cols) {
              const int ex = er + ce[c] - shift;
              const int64_t o = jb.out_off + r + (int64_t)cc * jb.ld;
              if (MODE == MODE_T) {
                Th[o] = ldexp_f(hi[g * 8 + c], ex);
                Tl[o] = ldexp_f(lo[g * 8 + c], ex);
              } else {
                F[o] += ldexp((double)hi[g * 8 + c] + (double)lo[g * 8 + c], ex);
              }
            }
          }
        }
      }
    }
    if (!ok) {
      abort_flag = 1;
      atomicExch(status, 4);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

}  // namespace sp
}  // namespace su2
