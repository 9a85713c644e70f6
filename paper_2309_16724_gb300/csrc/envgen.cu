// Device generation of synthetic-entry operator blocks with the same
// counter-based generator as the host code (SplitMix64, Steele, Lea, Flood
// 2014): element idx of a block with key k is mix64(k + (idx+1) * gamma)
// mapped to [-1, 1) by (x >> 11) * 2^-53 * 2 - 1, then scaled.  Every value
// is produced by the same IEEE operations as on the host, so both agree bit
// for bit.
#include <cuda_runtime.h>

#include "su2_internal.h"

namespace su2 {
namespace {

__device__ __forceinline__ uint64_t dmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double duniform(uint64_t key, uint64_t idx) {
  const uint64_t x = dmix64(key + (idx + 1) * 0x9E3779B97F4A7C15ull);
  return __dmul_rn(double(x >> 11), 1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// one CTA per (block, 64K-element slab)
__global__ void gen_kernel(const GenBlock* __restrict__ gb, const int64_t* __restrict__ unit_block,
                           const int64_t* __restrict__ unit_start, double* __restrict__ arena, int adjoint_pass) {
  const GenBlock g = gb[unit_block[blockIdx.x]];
  if ((g.kind == 2) != (adjoint_pass != 0)) return;
  const int64_t n = int64_t(g.rows) * g.cols;
  const int64_t i0 = unit_start[blockIdx.x];
  const int64_t i1 = i0 + 65536 < n ? i0 + 65536 : n;
  double* m = arena + g.off;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const int r = int(i % g.rows), c = int(i / g.rows);
    if (g.kind == 0) {
      m[i] = __dmul_rn(duniform(g.key, uint64_t(i)), g.scale);
    } else if (g.kind == 1) {
      const double x = __dmul_rn(duniform(g.key, uint64_t(i)), g.scale);
      const double y = __dmul_rn(duniform(g.key, uint64_t(c) + uint64_t(r) * g.rows), g.scale);
      double v = __dmul_rn(0.1, __dadd_rn(x, y));
      if (r == c) v = __dadd_rn(v, __ddiv_rn(2.0 * r, double(g.rows)));
      m[i] = v;
    } else {
      // adjoint: base block is cols x rows
      m[i] = __dmul_rn(g.scale, arena[g.base_off + c + int64_t(r) * g.cols]);
    }
  }
}

}  // namespace

// returns a CUDA error code (0 on success)
int generate_side(const SideOps& so, double* d_arena, cudaStream_t s) {
  if (so.gen.empty()) return 0;
  std::vector<int64_t> ub, us;
  for (size_t b = 0; b < so.gen.size(); ++b) {
    const int64_t n = int64_t(so.gen[b].rows) * so.gen[b].cols;
    for (int64_t i = 0; i < n; i += 65536) {
      ub.push_back(int64_t(b));
      us.push_back(i);
    }
  }
  GenBlock* dg = nullptr;
  int64_t *dub = nullptr, *dus = nullptr;
  cudaError_t e = cudaMalloc(&dg, so.gen.size() * sizeof(GenBlock));
  if (e == cudaSuccess) e = cudaMalloc(&dub, ub.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&dus, us.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMemcpy(dg, so.gen.data(), so.gen.size() * sizeof(GenBlock), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dub, ub.data(), ub.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dus, us.data(), us.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !ub.empty()) {
    gen_kernel<<<unsigned(ub.size()), 256, 0, s>>>(dg, dub, dus, d_arena, 0);
    gen_kernel<<<unsigned(ub.size()), 256, 0, s>>>(dg, dub, dus, d_arena, 1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaFree(dg);
  cudaFree(dub);
  cudaFree(dus);
  return int(e);
}

}  // namespace su2
