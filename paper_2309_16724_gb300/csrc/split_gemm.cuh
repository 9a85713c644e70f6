// Persistent split-precision stripe GEMM on tcgen05 (sm_103a).
//
// Operands are pre-tiled "slabs": an R x K FP64 matrix (R = M or N side,
// K-major) cut into S BF16 slices, stored as sub-tiles of up to 128 rows x
// 16 K in the UMMA no-swizzle K-major core-matrix layout (core matrix
// (mi, ki) at (mi*2 + ki)*128 bytes, row r%8 at 16*(r%8)); the compact layout
// (tile_rows / slab_pos below) stores a last row tile with only its rows,
// and the S slices of consecutive 16-K steps of a row tile follow each other,
// so one bulk copy per operand fills a pipeline stage.  Slice i holds
// q_i * 2^-8i where q_i are the integers peeled from x * 2^(8 - sigma_row)
// (|x| < 2^sigma_row): |q_0| <= 256, |q_i| <= 128.
//
// One job = one 128 x 128 output tile and a list of items (A slab, B slab,
// K steps); all items of a job share the row and column scales, so the
// K-concatenated stripe sum_items A_item . B_item^T accumulates in TMEM
// without a separate reduction (the stripe product of Sec. III.A).  Slice
// pairs (i, j), i + j < S, go to four FP32 TMEM accumulators of 128 columns
// (all 512) by level l = min(i + j, 3).  Levels 0, 1 and 2 hold integer
// multiples of their unit 2^-8l below 2^24 for K chunks of 192 (level 2 grows
// by at most 2*256*128 + 128^2 = 2^16.3 per K, 192 K give 2^23.9), hence are
// exact whatever rounding the tensor core applies when it adds into the
// accumulator (it truncates: a shared tail accumulator of many pairs would
// collect a biased error of order #adds * 2^-23 of its size); level 3 carries
// the 2^-24-weighted tail.  A chunk is up to 192 K of one item; after it the
// drain warps fold the four levels into a float-float register accumulator
// (K2: scaled by the item's per-column factor, so every task keeps its own
// S*8 bits), and the first MMA of the next chunk into each level overwrites
// it.  The chunk enters as the exact pair (x0 + r, (y1 - r) + y2 + y3), with
// r = rint(y1): level 0 is an integer of at most 192 * 2^16 and level 1 stays
// below 2^16, so x0 + r is an integer below 2^24 and y1 - r is at most 1/2.
// The job's first chunk becomes the accumulator; later ones are added with
// TwoSum and renormalised.  At the end of the job they write the tile (K1:
// normalised float-float T; K2: F += FP64).
//
// Warp roles (576 threads): warp 0, one lane: job fetcher (dynamic schedule:
// an atomic job counter, handed to the drain warps through a shared-memory
// ring) and bulk-copy producer, which leaves one metadata word per stage for
// the MMA issuer; warp 1: MMA issuer, reading shared memory only (the
// converged warp runs the loop, one elected lane issues each MMA);
// warps 2..17: drain and epilogue (TMEM lane quarter w%4; the job's columns
// are split evenly among the four warps of a quarter).  The drain warps
// arrive on barriers with one lane each.
// Every mbarrier wait is bounded; on timeout the CTA records a status,
// stops issuing, waits (bounded) for its own copies and MMAs, frees TMEM and
// returns.  The waits of the work loops poll at most `spin` times (a launch
// argument, normally kSpinLimit); the final waits for the CTA's own copies
// and MMAs always use kSpinLimit.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace su2 {
namespace sp {

constexpr int kRows = 128;           // M tile; slab row tile
// One TMEM accumulator buffer of 128-column job tiles: the drain of a chunk
// stalls the MMAs.  Two buffers of 64-column tiles (drain overlapped) were
// measured slower: in place an MMA costs about the same time for N = 64 and
// N = 128, so the wide tile does twice the work per MMA.
constexpr int kNumBuf = 1;
constexpr int kCols = 128;  // N tile of a job
constexpr int kKS = 16;              // K per pipeline stage (one MMA K step)
constexpr int kSub = kRows * kKS * 2;  // bytes of one 128 x 16 BF16 sub-tile (slabs, A stage)
constexpr int kSubB = kCols * kKS * 2;  // bytes of the B part of a stage slice (kCols rows)
constexpr int kBufCols = 4 * kCols;  // TMEM columns of one accumulator buffer (4 levels)
constexpr int kDrainCols = kCols / 4;  // most columns per drain thread (16 drain warps: 4 lane quarters x 4 groups)
constexpr int kGroup = kDrainCols >= 32 ? 4 : 8;  // columns per TMEM load group
constexpr int kMaxS = 6;
constexpr int kChunkSteps = 12;      // 16-K steps per exact drain chunk (192 K)
constexpr int kLead = 8;             // leading slice |q_0| <= 2^kLead, the others |q_i| <= 128
constexpr int kRing = 4;             // job ring slots
constexpr int kMaxStages = 8;
// A pipeline stage holds sk consecutive 16-K steps (sk divides kChunkSteps;
// a tile-shape parameter chosen by the autotuner): S A slices of up to 128
// rows and S B slices of up to kCols rows per step
__host__ __device__ constexpr int stage_bytes_of(int S, int sk) { return sk * S * (kSub + kSubB); }
// stages that fit in 220 KB of shared memory (at most kMaxStages)
__host__ __device__ constexpr int stages_of(int S, int sk) {
  return (225280 / stage_bytes_of(S, sk)) < kMaxStages ? (225280 / stage_bytes_of(S, sk)) : kMaxStages;
}
constexpr int kSmemMax = 225280 + 1024;  // largest dynamic shared memory of a launch (+ 1 KB for alignment)
__host__ __device__ constexpr bool stage_k_valid(int S, int sk) {
  return sk >= 1 && sk <= 6 && kChunkSteps % sk == 0 && stages_of(S, sk) >= 2;
}
// per-stage word the producer leaves for the MMA issuer (no global loads on
// the issue path); bits 4..7: 16-K steps in the stage, bits 8..11: MMA N / 16,
// bits 12..15: stored A rows / 16
enum : uint32_t { kMetaFirst = 1, kMetaLast = 2, kMetaEnd = 8 };

// Compact slab layout: row tile tr of an R-row operand stores only its rows,
// rounded up to 16; its (16-K step k, slice i) sub-tile sits at
// tr * kst * S * kSub + (k * S + i) * tile_rows * 32 (core matrices of 8 rows x
// 16 bytes, (mi * 2 + ki) * 128 within the sub-tile).  All tiles but the last
// hold 128 rows.
__host__ __device__ inline int tile_rows(int R, int tr) {
  const int r = R - tr * kRows;
  return ((r < kRows ? r : kRows) + 15) & ~15;
}
__host__ __device__ inline int64_t slab_pos(int R, int kst, int S, int tr, int k, int i) {
  return int64_t(tr) * kst * S * kSub + (int64_t(k) * S + i) * tile_rows(R, tr) * 32;
}
constexpr int kDrainWarps = 16;
constexpr int kThreads = 64 + 32 * kDrainWarps;  // producer + MMA + drain warps
constexpr long kSpinLimit = 1L << 26;

struct Item {
  int64_t a_off, b_off;  // byte offsets of the item's A / B row tiles in their compact slabs
  int32_t nst;           // K stages of 16
  int32_t pad;
  int64_t sc_off;        // MODE_F: offset of the item's per-column drain exponents (a multiple of 128), -1 otherwise
};
// MODE_F: task t's B slab is cut relative to its own column exponents; the
// drain multiplies each chunk of t by 2^d, d = own(col) - gamma(col) in
// [-126, 0] (an exact power of two, <= 1), before adding it to the tile
// accumulator.  dexp[sc_off + col] holds the biased exponent 127 + d, the
// exponent field of the FP32 number 2^d, or 0 (the factor 0) for a column
// that is zero.  The per-task vector is padded to whole 128-column tiles.
struct TaskScale {
  const uint8_t* dexp;
};
// A job computes an M x N tile of the product; the MMA's M side (TMEM
// lanes) comes from the items' a_off slabs and its N side (TMEM columns) from
// the b_off slabs.  Without kJobTrans the M side runs along the output
// block's rows; with it the tile is computed transposed (M along the output
// columns, N along its rows) and the A and B slab arrays swap roles.  The
// host picks per output block the orientation with the smaller modelled cost
// (M is always 128 rows; N is the valid extent rounded up to 16).  The
// element of lane p and TMEM column q is written at out_off + p + q * ld, or
// with kJobLaneStride at out_off + p * ld + q (a transposed tile of a
// column-major block; a transposed tile of a row-major block needs no flag).
constexpr int32_t kJobTrans = 1;
constexpr int32_t kJobLaneStride = 2;
struct Job {
  int64_t out_off;       // element offset of the output block (column-major, leading dimension ld)
  int32_t rows, cols;    // valid extent along M and along N (the block's rows and columns, swapped if transposed)
  int32_t ld, tr, tc;    // leading dimension of the block; tile indices along M (kRows) and N (kCols)
  int32_t i0, i1;        // items
  int32_t rsc, csc;      // offsets of the exponent arrays of the block's rows / columns
  int32_t nst;           // total K stages of all items
  int32_t nmma;          // MMA N of this tile: the valid N extent rounded up to 16 (<= kCols)
  int32_t flags;         // kJobTrans, kJobLaneStride
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

// bounded wait of the work loops (at most `limit` polls, a launch argument:
// kSpinLimit unless the caller shortened it); false on timeout or when
// another role aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int limit) {
  for (int it = 0; it < limit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  return false;
}

// bounded wait by every lane of a warp, then a warp vote: the warp leaves
// converged (the .sync.aligned TMEM loads that follow need that) and agrees
// on the outcome (polling by lane 0 alone measured slower)
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int limit) {
  const bool got = mbar_wait(bar, parity, abort_flag, limit);
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

// D (+)= A * B^T; ACC = false overwrites D.  Called by all 32 lanes of the
// MMA warp with the same operands; one lane, chosen by elect.sync, issues
// the MMA.  (Issued by a lone lane in a divergent branch, an MMA measured
// about 75 cycles at any N; from the converged warp 67 cycles at N = 128 and
// 53 at N = 64, close to the tensor core's own 64 and 48.)
template <bool ACC>
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc) {
  if (ACC)
    asm volatile(
        "{\n.reg .pred p;\nelect.sync _|p, 0xffffffff;\n"
        "@p tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc));
  else
    asm volatile(
        "{\n.reg .pred p;\nelect.sync _|p, 0xffffffff;\n"
        "@p tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 0;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc));
}

// the S(S+1)/2 slice products of one 16-K step, unrolled: pair (i, j) goes to
// level min(i + j, 3) (kCols TMEM columns each from tbuf); da / db describe
// slice 0 of A / B, slice i sits as16 / bs16 16-byte units further (the
// descriptor's address field counts 16-byte units; an A slice stored with
// fewer than 128 rows lets the MMA read the next slice's bytes as rows past
// the tile, whose outputs are never used).  In the first step of a chunk the
// first product into each level, (0, level), overwrites it.
template <int S, bool FIRST>
__device__ __forceinline__ void issue_stage(uint32_t tbuf, uint64_t da, uint64_t db, uint32_t as16, uint32_t bs16,
                                            uint32_t idesc) {
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int jj = 0; jj < S - i; ++jj) {
      const int lvl = (i + jj) < 3 ? (i + jj) : 3;
      const uint64_t a = da + (uint64_t)(i * as16);
      const uint64_t b = db + (uint64_t)(jj * bs16);
      if (FIRST && i == 0 && jj == lvl) mma_bf16<false>(tbuf + lvl * kCols, a, b, idesc);
      else mma_bf16<true>(tbuf + lvl * kCols, a, b, idesc);
    }
}

// commit of the MMAs issued so far, by one elected lane of the converged MMA warp
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "{\n.reg .pred p;\nelect.sync _|p, 0xffffffff;\n"
      "@p tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(bar)
      : "memory");
}

// four 32x32b.x4 TMEM loads (four columns of each accumulator level) and
// the wait in one asm statement (see below)
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

// four 32x32b.x8 TMEM loads (eight columns of each accumulator level) and
// the wait in one asm statement: tcgen05.ld writes its destination registers
// asynchronously, so they must not exist as values in the program before
// tcgen05.wait::ld (a separate wait statement would let the compiler reuse or
// read them early)
__device__ __forceinline__ void tmem_ld8x4_wait(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                                float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%33];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%34];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%35];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// kG columns of all four accumulator levels (level l at column offset l * kCols)
template <int kG>
__device__ __forceinline__ void tmem_ld_levels(uint32_t a, float (&x)[4 * kG]);
template <>
__device__ __forceinline__ void tmem_ld_levels<4>(uint32_t a, float (&x)[16]) {
  tmem_ld4x4_wait(a, a + kCols, a + 2 * kCols, a + 3 * kCols, x);
}
template <>
__device__ __forceinline__ void tmem_ld_levels<8>(uint32_t a, float (&x)[32]) {
  tmem_ld8x4_wait(a, a + kCols, a + 2 * kCols, a + 3 * kCols, x);
}

// packed FP32 pairs (two drain columns per instruction); every step is the
// same IEEE operation on each half, so TwoSum stays error-free.  a - b is
// fma(b, -1, a): b * -1 is exact, so the one rounding gives RN(a - b) in a
// single packed instruction with no separate negation
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// x * 2^k: one multiply by the power of two built from its exponent field
// while 2^k is a normal number (the correctly rounded product, as ldexp
// gives), ldexp otherwise
__device__ __forceinline__ float ldexp_f(float x, int k) {
  return (k >= -126 && k <= 127) ? x * __int_as_float((127 + k) << 23) : ldexpf(x, k);
}
__device__ __forceinline__ double ldexp_d(double x, int k) {
  if (k >= -1022 && k <= 1023) return x * __longlong_as_double((long long)(1023 + k) << 52);
  k = max(-2044, min(2046, k));
  const int k1 = k / 2;
  return x * __longlong_as_double((long long)(1023 + k1) << 52) * __longlong_as_double((long long)(1023 + k - k1) << 52);
}

template <int MODE, int S>
__global__ void __launch_bounds__(kThreads, 1)
    split_gemm_kernel(const Job* __restrict__ jobs, int njobs, const Item* __restrict__ items,
                      const unsigned char* __restrict__ Aslab, const unsigned char* __restrict__ Bslab,
                      const int* __restrict__ rexp, const int* __restrict__ cexp, int shift,
                      float* __restrict__ Th, float* __restrict__ Tl, double* __restrict__ F, int* __restrict__ status,
                      int* __restrict__ job_counter, TaskScale ts, int sk, int spin) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int stage_bytes = stage_bytes_of(S, sk);
  const int NS = stages_of(S, sk);
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], accf_bar[2], acce_bar[2], done_bar;
  __shared__ __align__(8) uint64_t jq_full[kRing], jq_empty[kRing];
  __shared__ int job_ring[kRing];
  __shared__ Job job_slot[kRing];  // the job itself: the drain reads its fields here when it needs them
  __shared__ uint32_t stage_meta[kMaxStages];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[s])));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf_bar[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce_bar[b])), "r"(kDrainWarps));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done_bar)));
    for (int r = 0; r < kRing; ++r) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&jq_full[r])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&jq_empty[r])), "r"(kDrainWarps));
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
  constexpr int nlev = S < 4 ? S : 4;
  if (warp == 0) {
    // ------------------------------------------------------------ producer
    // fetches jobs for the drain warps (job ring) and fills the stage ring
    // for the MMA issuer, with one metadata word per stage
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0;  // phase of the current use of slot st (flips when st wraps)
      int nissued = 0;
      bool ok = true;
      for (int k = 0; ok; ++k) {
        const int slot = k % kRing;
        if (!mbar_wait(smem_u32(&jq_empty[slot]), ((k / kRing) & 1) ^ 1, &abort_flag, spin)) {
          ok = false;
          break;
        }
        const int jnext = atomicAdd(job_counter, 1);
        const int j = jnext < njobs ? jnext : -1;
        Job jb{};
        if (j >= 0) {
          jb = jobs[j];
          job_slot[slot] = jb;
        }
        job_ring[slot] = j;
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&jq_full[slot])) : "memory");
        if (j < 0) break;
        const bool jtrans = (jb.flags & kJobTrans) != 0;
        const unsigned char* mslab = jtrans ? Bslab : Aslab;  // M side (TMEM lanes)
        const unsigned char* nslab = jtrans ? Aslab : Bslab;  // N side (TMEM columns)
        const int arows = tile_rows(jb.rows, jb.tr);
        const int abytes = arows * 32, bbytes = jb.nmma * 32;  // stored bytes of one A / B sub-tile
        const uint32_t nmeta = ((uint32_t)(jb.nmma >> 4) << 8) | ((uint32_t)(arows >> 4) << 12);
        for (int it = jb.i0; it < jb.i1 && ok; ++it) {
          const Item item = items[it];
          const int nstage = (item.nst + sk - 1) / sk;
          for (int ks = 0; ks < nstage; ++ks) {
            if (!mbar_wait(smem_u32(&empty_bar[st]), ph ^ 1, &abort_flag, spin)) {
              ok = false;
              break;
            }
            const int k16 = ks * sk;  // first 16-K step of the stage within the item
            const int nk = min(sk, item.nst - k16);
            uint32_t m = nmeta | ((uint32_t)nk << 4);
            if (k16 % kChunkSteps == 0) m |= kMetaFirst;
            if ((k16 + sk) % kChunkSteps == 0 || ks == nstage - 1) m |= kMetaLast;
            stage_meta[st] = m;
            const uint32_t fb = smem_u32(&full_bar[st]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                         "r"(nk * S * (abytes + bbytes))
                         : "memory");
            // the nk steps x S slices of A, then of B, are contiguous in their slabs
            const uint32_t dst = smem_u32(smem + st * stage_bytes);
            const unsigned char* srcA = mslab + item.a_off + (int64_t)k16 * S * abytes;
            const unsigned char* srcB = nslab + item.b_off + (int64_t)k16 * S * bbytes;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                "l"(srcA), "r"(nk * S * abytes), "r"(fb)
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    dst + sk * S * kSub),
                "l"(srcB), "r"(nk * S * bbytes), "r"(fb)
                : "memory");
            ++nissued;
            if (++st == NS) {
              st = 0;
              ph ^= 1;
            }
          }
        }
      }
      // end marker for the MMA issuer: a stage without data
      if (ok) {
        if (mbar_wait(smem_u32(&empty_bar[st]), ph ^ 1, &abort_flag, spin)) {
          stage_meta[st] = kMetaEnd;
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full_bar[st])) : "memory");
          ++nissued;
          if (++st == NS) {
            st = 0;
            ph ^= 1;
          }
        } else {
          ok = false;
        }
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(status, 4);
      }
      // wait (bounded) for the last use of every slot: all copies this CTA issued have landed
      for (int b = 0; b < NS && b < nissued; ++b) {
        int s2 = st - 1 - b;
        uint32_t p2 = ph;
        if (s2 < 0) {
          s2 += NS;
          p2 ^= 1;
        }
        bool fin = false;
        for (long it = 0; it < kSpinLimit && !fin; ++it) fin = mbar_try(smem_u32(&full_bar[s2]), p2);
        if (!fin) atomicExch(status, 4);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    // reads only shared memory: the stage ring and its metadata words.  The
    // whole warp runs the loop (its values are warp-uniform); one elected
    // lane issues each MMA and commit.
    {
      int st = 0;
      uint32_t ph = 0;
      uint32_t chunk = 0;  // chunk c accumulates in TMEM buffer c % kNumBuf
      bool ok = true;
      const uint32_t sbase = smem_u32(smem);
      for (;;) {
        if (!warp_wait(smem_u32(&full_bar[st]), ph, &abort_flag, spin)) {
          ok = false;
          break;
        }
        const uint32_t m = *(volatile uint32_t*)&stage_meta[st];
        if (m & kMetaEnd) break;
        const uint32_t buf = chunk % kNumBuf;
        if (m & kMetaFirst) {
          // the buffer's previous chunk (c - kNumBuf) must have been read by the drain
          if (!warp_wait(smem_u32(&acce_bar[buf]), ((chunk / kNumBuf) & 1) ^ 1, &abort_flag, spin)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
        }
        const uint32_t n16 = (m >> 8) & 0xf, a16 = (m >> 12) & 0xf;
        const uint32_t idesc = idesc_n((int)n16 * 16);
        const uint32_t bs16 = n16 * 32, as16 = a16 * 32;  // sub-tile strides in 16-byte units (rows * 32 / 16)
        const uint32_t sa = sbase + st * stage_bytes;
        const uint64_t da = make_desc(sa), db = make_desc(sa + sk * S * kSub);
        const uint32_t tb = tmem + buf * kBufCols;
        const int nk = (int)((m >> 4) & 0xf);
        if (m & kMetaFirst) issue_stage<S, true>(tb, da, db, as16, bs16, idesc);
        else issue_stage<S, false>(tb, da, db, as16, bs16, idesc);
        for (int kk = 1; kk < nk; ++kk)
          issue_stage<S, false>(tb, da + (uint64_t)(kk * S * as16), db + (uint64_t)(kk * S * bs16), as16, bs16, idesc);
        mma_commit(smem_u32(&empty_bar[st]));
        if (m & kMetaLast) {
          mma_commit(smem_u32(&accf_bar[buf]));
          chunk += 1;
        }
        if (++st == NS) {
          st = 0;
          ph ^= 1;
        }
      }
      if (!ok && lane == 0) {
        abort_flag = 1;
        atomicExch(status, 4);
      }
      // all MMAs issued by this warp complete before TMEM is released
      mma_commit(smem_u32(&done_bar));
      bool fin = false;
      for (long it = 0; it < kSpinLimit && !fin; ++it) fin = mbar_try(smem_u32(&done_bar), 0);
      if (!fin) atomicExch(status, 4);
    }
  } else {
    // ------------------------------------------------------------ drain / epilogue
    const int q = warp & 3;             // TMEM lane quarter
    const int cgrp = (warp - 2) >> 2;   // column group: a quarter of the job's MMA columns
    const int row = q * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    uint32_t chunk = 0;
    bool ok = true;
    for (int k = 0; ok; ++k) {
      const int slot = k % kRing;
      if (!warp_wait(smem_u32(&jq_full[slot]), (k / kRing) & 1, &abort_flag, spin)) {
        ok = false;
        break;
      }
      const int j = job_ring[slot];
      if (j < 0) {
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&jq_empty[slot])) : "memory");
        break;
      }
      // the job stays in its ring slot until this warp's epilogue is done; its
      // fields are read from shared memory where they are used, so that they
      // hold no registers across the chunk loop
      const volatile Job& jb = job_slot[slot];
      // float-float tile accumulator (leading, trailing part), set by the
      // job's first chunk
      float2 hi2[kDrainCols / 2], lo2[kDrainCols / 2];
#pragma unroll
      for (int c = 0; c < kDrainCols / 2; ++c) {
        hi2[c] = make_float2(0.f, 0.f);
        lo2[c] = make_float2(0.f, 0.f);
      }
      bool first = true;
      // the 16 drain warps split the job's nmma columns evenly: nmma / 4 (a
      // multiple of 4, at most kDrainCols) per lane-quarter warp, so a narrow
      // tile drains in proportionally less time
      constexpr int kNG = kDrainCols / kGroup;
      static_assert(kGroup == 4, "the drain exponent of column 4g + c is byte c of word g");
      const int w = jb.nmma >> 2;
      const int ng = w / kGroup;  // column groups of this warp
      const int c0 = jb.tc * kCols + cgrp * w;
      const uint32_t lane_addr = lane_base + cgrp * w;
      const int i1 = jb.i1;
      const bool trans = (jb.flags & kJobTrans) != 0;
      const int p = jb.tr * kRows + row;  // this lane's index along M
      for (int it = jb.i0; it < i1 && ok; ++it) {
        const Item item = items[it];
        // MODE_F: the item's drain exponents (one per output column), fetched
        // before the chunk wait.  Output columns along N: the same for every
        // lane, so lane v holds word v (bytes = columns 4v .. 4v + 3) and the
        // group loop broadcasts it.  Transposed: the lane's own column, its
        // byte replicated into all four positions.
        uint32_t dxl = 0u;
        if (MODE == MODE_F) {
          if (trans) {
            dxl = (uint32_t)__ldg(ts.dexp + item.sc_off + p) * 0x01010101u;
          } else {
            const uint32_t* dw = reinterpret_cast<const uint32_t*>(ts.dexp + item.sc_off + c0);
            if (lane < ng) dxl = __ldg(dw + lane);
          }
        }
        const int nch = (item.nst + kChunkSteps - 1) / kChunkSteps;
        for (int ch = 0; ch < nch; ++ch) {
          const uint32_t buf = chunk % kNumBuf;
          if (!warp_wait(smem_u32(&accf_bar[buf]), (chunk / kNumBuf) & 1, &abort_flag, spin)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
          for (int g = 0; g < kNG; ++g) {
            if (g >= ng) break;
            const uint32_t a = lane_addr + buf * kBufCols + g * kGroup;
            float x[4 * kGroup];  // levels 0..3, kGroup columns each
            tmem_ld_levels<kGroup>(a, x);
            const uint32_t dxg = MODE == MODE_F ? __shfl_sync(0xffffffffu, dxl, trans ? lane : g) : 0u;
            if (g == ng - 1) {
              // the warp's last TMEM read of this chunk has completed: hand
              // the buffer back before the arithmetic on the last group
              asm volatile("tcgen05.fence::before_thread_sync;");
              __syncwarp();
              if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[buf])) : "memory");
            }
#pragma unroll
            for (int c = 0; c < kGroup; c += 2) {
              const int k = g * kGroup + c;  // column within this thread's group (even)
              const float2 z = make_float2(0.f, 0.f);
              const float2 x0 = make_float2(x[c], x[c + 1]);
              const float2 y1 = nlev > 1 ? make_float2(x[kGroup + c], x[kGroup + c + 1]) : z;
              const float2 y2 = nlev > 2 ? make_float2(x[2 * kGroup + c], x[2 * kGroup + c + 1]) : z;
              const float2 y3 = nlev > 3 ? make_float2(x[3 * kGroup + c], x[3 * kGroup + c + 1]) : z;
              // x0 + y1 split exactly without TwoSum: level 0 is an integer
              // with |x0| <= 192 * 256 * 256 (slice 0 of each operand is an
              // integer of magnitude <= 256), level 1 a multiple of 2^-8 with
              // |y1| <= 192 * 2 * 256 * 128 * 2^-8 < 2^22, so r = rint(y1) (by
              // the 1.5 * 2^23 shift), s = x0 + r (an integer < 2^24) and
              // e = y1 - r (|e| <= 1/2) are all exact and s + e = x0 + y1
              const float2 mg = make_float2(12582912.f, 12582912.f);
              const float2 r = sub2(add2(y1, mg), mg);
              float2 sc = add2(x0, r);
              float2 t = add2(sub2(y1, r), add2(y2, y3));
              if (MODE == MODE_F) {
                // 2^d of columns k and k + 1: the biased exponent byte moved
                // to the FP32 exponent field (byte 3 of a word, shifted right
                // once); the scaling of both parts is exact
                const uint32_t b0 = __byte_perm(dxg, 0u, 0x0444u | ((uint32_t)c << 12)) >> 1;
                const uint32_t b1 = __byte_perm(dxg, 0u, 0x0444u | ((uint32_t)(c + 1) << 12)) >> 1;
                const float2 f2 = make_float2(__uint_as_float(b0), __uint_as_float(b1));
                sc = __fmul2_rn(sc, f2);
                t = __fmul2_rn(t, f2);
              }
              if (first) {  // the accumulator is zero: it becomes the chunk (sc, t)
                hi2[k >> 1] = sc;
                lo2[k >> 1] = t;
              } else {  // TwoSum into the leading part, the rest into the trailing part, renormalise
                float2 h, e2;
                two_sum2(hi2[k >> 1], sc, h, e2);
                const float2 l = add2(lo2[k >> 1], add2(e2, t));
                const float2 hs = add2(h, l);
                lo2[k >> 1] = sub2(l, sub2(hs, h));
                hi2[k >> 1] = hs;
              }
            }
          }
          if (ng <= 0) {  // (nmma >= 16 gives ng >= 1; kept so that the barrier always completes)
            __syncwarp();
            if (lane == 0)
              asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce_bar[buf])) : "memory");
          }
          first = false;
          chunk += 1;
        }
      }
      if (!ok) break;
      // epilogue: scale by 2^(rexp(block row) + cexp(block column) - shift)
      // and write; lane index p along M, column index q along N, the block
      // element (p, q), or (q, p) when transposed
      const int jrows = jb.rows, jcols = jb.cols, jld = jb.ld;
      if (p < jrows) {
        const int ep = trans ? cexp[jb.csc + p] : rexp[jb.rsc + p];
        const int* const eq = trans ? rexp + jb.rsc : cexp + jb.csc;
        const bool lstride = (jb.flags & kJobLaneStride) != 0;
        const int64_t obase = jb.out_off + (lstride ? (int64_t)p * jld : (int64_t)p);
        const int64_t ostep = lstride ? 1 : jld;
#pragma unroll
        for (int c = 0; c < kDrainCols; ++c) {
          if (c >= w) break;
          const int q = c0 + c;
          if (q < jcols) {
            const int ex = ep + eq[q] - shift;
            const int64_t o = obase + (int64_t)q * ostep;
            if (MODE == MODE_T) {
              // a job whose only chunk was its first leaves (hi, lo) not
              // normalised; T goes out normalised (TwoSum), since the column
              // exponents of T are taken from its leading part alone
              const float ha = (c & 1) ? hi2[c >> 1].y : hi2[c >> 1].x;
              const float la = (c & 1) ? lo2[c >> 1].y : lo2[c >> 1].x;
              const float hs = __fadd_rn(ha, la), bb = __fsub_rn(hs, ha);
              const float ls = __fadd_rn(__fsub_rn(ha, __fsub_rn(hs, bb)), __fsub_rn(la, bb));
              Th[o] = ldexp_f(hs, ex);
              Tl[o] = ldexp_f(ls, ex);
            } else {
              F[o] += ldexp_d((double)((c & 1) ? hi2[c >> 1].y : hi2[c >> 1].x) +
                                (double)((c & 1) ? lo2[c >> 1].y : lo2[c >> 1].x),
                            ex);
            }
          }
        }
      }
      // the job's ring slot may now take the next job
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&jq_empty[slot])) : "memory");
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
