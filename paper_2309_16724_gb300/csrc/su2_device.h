// Library state shared by the host API and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "su2_internal.h"

// FP64 path: 64x64 output tiles.
namespace su2 {
constexpr int kTile = 64;

// K1: T(k1 x n) = E(k1 x k2) . D(n x k2)^T for one deduplicated
// (right operator block, input block) pair, one 64x64 tile of T.
struct K1Job {
  int64_t e_off, d_off, t_off;
  int32_t k1, k2, n, tr, tc, pad;
};
// K2: one 64x64 tile of an output block F{f}, summed over the tasks
// [t0, t1) of the current chunk that write into f (output stationary).
struct K2Job {
  int64_t f_off;
  int32_t m, n, tr, tc, t0, t1;
};
enum { K2_A_IDENTITY = 1, K2_B_FROM_PSI = 2 };
struct K2Task {
  int64_t a_off;  // left operator block in the left arena (m x k1), unused for identity
  int64_t b_off;  // T in the chunk buffer (k1 x n) or the input block of psi
  int32_t k1, flags;
  double v;       // sector-value table entry
};
struct DiagJob {  // one output block of the diagonal, its diagonal tasks [t0, t1)
  int64_t f_off;
  int32_t m, n, t0, t1;
};
struct DiagTask {
  int64_t a_off, d_off;  // -1: identity
  int32_t lda, ldd;
  double v;
};
struct Chunk {
  int64_t k1_begin, k1_end, k2_begin, k2_end;
  double k1_flops, k2_flops;
};

// CUDA-event profiling of the hot-path launches
constexpr int kProfKinds = 6;  // kind 5 counts every hot-path kernel launch
struct Profiler {
  bool on = false;
  struct Pending { int kind; cudaEvent_t a, b; double flops; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  int64_t launches[kProfKinds] = {};
  double ms[kProfKinds] = {};
  double flops[kProfKinds] = {};
  cudaEvent_t get() {
    cudaEvent_t e;
    if (!pool.empty()) { e = pool.back(); pool.pop_back(); }
    else cudaEventCreate(&e);
    return e;
  }
  // returns the pending slot; call end() after the launch
  void count(int n) { launches[5] += n; }
  int begin(cudaStream_t s, int kind, double fl) {
    if (!on) return -1;
    Pending p{kind, get(), get(), fl};
    cudaEventRecord(p.a, s);
    pending.push_back(p);
    return int(pending.size()) - 1;
  }
  void end(cudaStream_t s, int slot) {
    if (slot >= 0) cudaEventRecord(pending[slot].b, s);
  }
  void drain() {
    for (auto& p : pending) {
      cudaEventSynchronize(p.b);
      float t = 0.f;
      cudaEventElapsedTime(&t, p.a, p.b);
      ms[p.kind] += t;
      launches[p.kind] += 1;
      flops[p.kind] += p.flops;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void reset() {
    drain();
    for (int i = 0; i < kProfKinds; ++i) { launches[i] = 0; ms[i] = 0; flops[i] = 0; }
  }
  ~Profiler() {
    for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// tasks whose four dimensions are all at most kSmallDim run in FP64 on CUDA
// cores in the split path (the small-task class)
constexpr int kSmallDim = 16;

void launch_heff_fp64(cudaStream_t s, const double* L, const double* R, const double* psi, double* F, double* T,
                      const K1Job* k1, const K2Job* k2, const K2Task* tasks, const Chunk& c, int64_t psi_len,
                      Profiler* prof);
void launch_diag(cudaStream_t s, const double* L, const double* R, double* d, const DiagJob* jobs, int64_t njobs,
                 const DiagTask* tasks, int64_t psi_len);
}  // namespace su2

namespace su2 {
// Out-of-core operator arenas (Sec. III.E-F).  The operator blocks of both
// sides share one logical arena laid out by the planner: [0, prefix) is
// resident on the device (blocks shared by several term chunks, blocks of
// the diagonal and of the small-task class, then the blocks of the first
// chunks up to the device budget), the rest lies in pinned host memory with
// the blocks of each chunk contiguous, [hs[c], he[c]).  Per H.psi the
// streamed range of chunk c is copied on a dedicated IO stream into device
// slot c % 2 while other chunks compute; events order each copy after the
// last reader of its slot and each chunk after its copy.
struct OpStream {
  bool on = false;
  std::vector<int> starts;       // term chunk boundaries (shared by the FP64 and split plans)
  int64_t prefix = 0;            // doubles resident on the device
  int64_t total = 0;             // doubles of the logical arena
  std::vector<int64_t> hs, he;   // streamed range of each chunk (logical offsets)
  int64_t slot = 0;              // doubles per device slot
  double* dbuf = nullptr;        // device: [0, prefix) resident, then the two slots
  double* host = nullptr;        // pinned host memory: logical [prefix, total)
  cudaStream_t io = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, join = nullptr;
  double io_bytes = 0.0;         // bytes copied per H.psi
  // the diagonals of the blocks the diagonal of H_eff reads (device, kept):
  // block b of side sd has its diagonal at ddiag[dg_off[sd][b]] (-1: none)
  std::vector<int64_t> dg_off[2];
  int64_t dg_total = 0;
  double* ddiag = nullptr;
  // device offset of a block at logical offset `off` read by chunk c
  int64_t dev_off(int64_t off, int c) const {
    return off < prefix ? off : prefix + int64_t(c & 1) * slot + (off - hs[size_t(c)]);
  }
};
}  // namespace su2

struct su2_ctx {
  int device = -1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int* d_status = nullptr;
};

struct su2_sectors {
  int site_kind = 0, N = 0, twoS = 0;
  std::vector<su2::Sector> left, right;
  std::vector<su2::Block> blocks;
  std::vector<su2_block> pub;
  int64_t psi_len = 0;
};

struct su2_env {
  su2_ctx* ctx = nullptr;
  int device = -1;  // the context's device, kept here so that destroying the
                    // environment never reads its context (which the caller
                    // may already have destroyed)
  su2::OpTable table;
  su2::SideOps L, R;
  std::vector<su2::Task> tasks;
  su2_env_info info{};
  int64_t psi_len = 0;
  std::vector<su2::Block> blocks;   // psi blocks
  std::vector<su2::Sector> lsec, rsec;
  int64_t split_budget = 0;
  int spin_limit = 0;  // polls of each work-loop wait of the split GEMM (0: the kernel's default)
  // FP64 plan
  std::vector<su2::Chunk> chunks;
  std::vector<su2::K1Job> k1;
  std::vector<su2::K2Job> k2;
  std::vector<su2::K2Task> k2t;
  std::vector<su2::DiagJob> dj;
  std::vector<su2::DiagTask> dt;
  int64_t t_elems = 0;  // T buffer size (doubles)
  // device copies
  double *dL = nullptr, *dR = nullptr, *dT = nullptr;
  su2::K1Job* dk1 = nullptr;
  su2::K2Job* dk2 = nullptr;
  su2::K2Task* dk2t = nullptr;
  su2::DiagJob* ddj = nullptr;
  su2::DiagTask* ddt = nullptr;
  double *d_in_scratch = nullptr, *d_out_scratch = nullptr;  // for host-buffer calls
  void* split = nullptr;  // split-precision state (opaque)
  su2::OpStream os;       // out-of-core operator arenas (os.on)
  su2::Profiler prof;
};
