// Native-FP64 path of H.psi (Eq. 2 over the sector-task-table of Eq. 3).
// K1 forms T = E . D^T for each deduplicated (right operator block, input
// block) of a chunk of operator-table rows; K2 is output stationary: one
// CTA owns a 64x64 tile of an output block F{f} and runs through every task
// of the chunk that writes into f, accumulating sum_t v_t A_t . T_t in
// registers (the K-concatenated stripe product, Sec. III.A, with no separate
// reduction step).  Deterministic: no atomics.
#include "su2_device.h"

namespace su2 {
namespace {

constexpr int TK = 16;
constexpr int NT = 256;

// acc += alpha * A(r0:r0+64, 0:K) . B(0:K, c0:c0+64); A column-major (lda),
// B(kk, c) = BT ? B[c + kk*ldb] : B[kk + c*ldb].  Out-of-range entries are 0.
template <bool BT>
__device__ __forceinline__ void tile_gemm(double (&acc)[4][4], const double* __restrict__ A, int lda,
                                          const double* __restrict__ B, int ldb, int M, int N, int K, int r0, int c0,
                                          double alpha, double (*sA)[kTile], double (*sB)[kTile]) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int k0 = 0; k0 < K; k0 += TK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = tid + NT * i;
      const int r = idx & 63, kk = idx >> 6;
      const int gr = r0 + r, gk = k0 + kk;
      sA[kk][r] = (gr < M && gk < K) ? alpha * A[gr + int64_t(gk) * lda] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = tid + NT * i;
      int kk, c;
      if (BT) {
        c = idx & 63;
        kk = idx >> 6;
      } else {
        kk = idx & 15;
        c = idx >> 4;
      }
      const int gc = c0 + c, gk = k0 + kk;
      double v = 0.0;
      if (gc < N && gk < K) v = BT ? B[gc + int64_t(gk) * ldb] : B[gk + int64_t(gc) * ldb];
      sB[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(NT) k1_fp64(const K1Job* __restrict__ jobs, const double* __restrict__ psi,
                                              const double* __restrict__ R, double* __restrict__ T) {
  __shared__ double sA[TK][kTile], sB[TK][kTile];
  const K1Job j = jobs[blockIdx.x];
  double acc[4][4] = {};
  const int r0 = j.tr * kTile, c0 = j.tc * kTile;
  tile_gemm<true>(acc, psi + j.e_off, j.k1, R + j.d_off, j.n, j.k1, j.n, j.k2, r0, c0, 1.0, sA, sB);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * jj;
      if (r < j.k1 && c < j.n) T[j.t_off + r + int64_t(c) * j.k1] = acc[i][jj];
    }
}

__global__ void __launch_bounds__(NT) k2_fp64(const K2Job* __restrict__ jobs, const K2Task* __restrict__ tasks,
                                              const double* __restrict__ L, const double* __restrict__ psi,
                                              const double* __restrict__ T, double* __restrict__ F) {
  __shared__ double sA[TK][kTile], sB[TK][kTile];
  const K2Job j = jobs[blockIdx.x];
  const int r0 = j.tr * kTile, c0 = j.tc * kTile;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int t = j.t0; t < j.t1; ++t) {
    const K2Task task = tasks[t];
    const double* B = ((task.flags & K2_B_FROM_PSI) ? psi : T) + task.b_off;
    if (task.flags & K2_A_IDENTITY) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * jj;
          if (r < j.m && c < j.n) acc[i][jj] = fma(task.v, B[r + int64_t(c) * task.k1], acc[i][jj]);
        }
    } else {
      tile_gemm<false>(acc, L + task.a_off, j.m, B, task.k1, j.m, j.n, task.k1, r0, c0, task.v, sA, sB);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * jj;
      if (r < j.m && c < j.n) F[j.f_off + r + int64_t(c) * j.m] += acc[i][jj];
    }
}

__global__ void diag_kernel(const DiagJob* __restrict__ jobs, const DiagTask* __restrict__ tasks,
                            const double* __restrict__ L, const double* __restrict__ R, double* __restrict__ d) {
  const DiagJob j = jobs[blockIdx.x];
  const int64_t n = int64_t(j.m) * j.n;
  for (int64_t x = threadIdx.x; x < n; x += blockDim.x) {
    const int r = int(x % j.m), c = int(x / j.m);
    double s = 0.0;
    for (int t = j.t0; t < j.t1; ++t) {
      const DiagTask tk = tasks[t];
      const double a = tk.a_off < 0 ? 1.0 : L[tk.a_off + r + int64_t(r) * tk.lda];
      const double b = tk.d_off < 0 ? 1.0 : R[tk.d_off + c + int64_t(c) * tk.ldd];
      s += tk.v * a * b;
    }
    d[j.f_off + x] = s;
  }
}

}  // namespace

void launch_heff_fp64(cudaStream_t s, const double* L, const double* R, const double* psi, double* F, double* T,
                      const K1Job* k1, const K2Job* k2, const K2Task* tasks, const Chunk& c, int64_t,
                      Profiler* prof) {
  const int64_t n1 = c.k1_end - c.k1_begin, n2 = c.k2_end - c.k2_begin;
  prof->count(int(n1 > 0) + int(n2 > 0));
  if (n1 > 0) {
    const int slot = prof->begin(s, 0, c.k1_flops);
    k1_fp64<<<unsigned(n1), NT, 0, s>>>(k1 + c.k1_begin, psi, R, T);
    prof->end(s, slot);
  }
  if (n2 > 0) {
    const int slot = prof->begin(s, 1, c.k2_flops);
    k2_fp64<<<unsigned(n2), NT, 0, s>>>(k2 + c.k2_begin, tasks, L, psi, T, F);
    prof->end(s, slot);
  }
}

void launch_diag(cudaStream_t s, const double* L, const double* R, double* d, const DiagJob* jobs, int64_t njobs,
                 const DiagTask* tasks, int64_t psi_len) {
  cudaMemsetAsync(d, 0, size_t(psi_len) * sizeof(double), s);
  if (njobs > 0) diag_kernel<<<unsigned(njobs), 256, 0, s>>>(jobs, tasks, L, R, d);
}

}  // namespace su2
