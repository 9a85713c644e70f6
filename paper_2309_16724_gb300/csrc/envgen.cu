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

// entry (r, c) of a generated block of `kind` (0 random, 1 HAM) with `rows` rows
__device__ __forceinline__ double gen_value(int kind, uint64_t key, double scale, int rows, int r, int c) {
  const uint64_t i = uint64_t(r) + uint64_t(c) * uint64_t(rows);
  if (kind == 0) return __dmul_rn(duniform(key, i), scale);
  const double x = __dmul_rn(duniform(key, i), scale);
  const double y = __dmul_rn(duniform(key, uint64_t(c) + uint64_t(r) * uint64_t(rows)), scale);
  double v = __dmul_rn(0.1, __dadd_rn(x, y));
  if (r == c) v = __dadd_rn(v, __ddiv_rn(2.0 * r, double(rows)));
  return v;
}

// one CTA per (block, 64K-element slab); block g is written at
// arena[g.off - shift]
__global__ void gen_kernel(const GenBlock* __restrict__ gb, const int64_t* __restrict__ unit_block,
                           const int64_t* __restrict__ unit_start, double* __restrict__ arena, int64_t shift) {
  const GenBlock g = gb[unit_block[blockIdx.x]];
  const int64_t n = int64_t(g.rows) * g.cols;
  const int64_t i0 = unit_start[blockIdx.x];
  const int64_t i1 = i0 + 65536 < n ? i0 + 65536 : n;
  double* m = arena + (g.off - shift);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const int r = int(i % g.rows), c = int(i / g.rows);
    if (g.kind == 2)  // adjoint: the base block is cols x rows, entry (c, r)
      m[i] = __dmul_rn(g.scale, gen_value(g.base_kind, g.key, g.base_scale, g.cols, c, r));
    else
      m[i] = gen_value(g.kind, g.key, g.scale, g.rows, r, c);
  }
}

}  // namespace

// Generates the blocks `which` of `gen` (all of them when which is null) into
// arena[off - shift]; returns a CUDA error code (0 on success).
int generate_blocks(const std::vector<GenBlock>& gen, const std::vector<int>* which, double* d_arena, int64_t shift,
                    cudaStream_t s) {
  std::vector<GenBlock> sel;
  if (which) {
    for (int b : *which) sel.push_back(gen[size_t(b)]);
  }
  const std::vector<GenBlock>& g = which ? sel : gen;
  if (g.empty()) return 0;
  std::vector<int64_t> ub, us;
  for (size_t b = 0; b < g.size(); ++b) {
    const int64_t n = int64_t(g[b].rows) * g[b].cols;
    for (int64_t i = 0; i < n; i += 65536) {
      ub.push_back(int64_t(b));
      us.push_back(i);
    }
  }
  GenBlock* dg = nullptr;
  int64_t *dub = nullptr, *dus = nullptr;
  cudaError_t e = cudaMalloc(&dg, g.size() * sizeof(GenBlock));
  if (e == cudaSuccess) e = cudaMalloc(&dub, ub.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&dus, us.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMemcpy(dg, g.data(), g.size() * sizeof(GenBlock), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dub, ub.data(), ub.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dus, us.data(), us.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !ub.empty()) {
    gen_kernel<<<unsigned(ub.size()), 256, 0, s>>>(dg, dub, dus, d_arena, shift);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaFree(dg);
  cudaFree(dub);
  cudaFree(dus);
  return int(e);
}

int generate_side(const SideOps& so, double* d_arena, cudaStream_t s) {
  return generate_blocks(so.gen, nullptr, d_arena, 0, s);
}

}  // namespace su2
