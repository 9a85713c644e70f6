// Out-of-core operator arenas (Sec. III.E "dedicated IO streams", Sec. III.F
// "dynamic memory buffer"): the operator blocks of an environment that does
// not fit on the device live partly in pinned host memory and are copied to
// the device per term chunk on an IO stream of their own, overlapped with the
// compute of other chunks.
//
// The paper's buffer serves a general task tree and evicts on demand.  The
// access pattern of H.psi is fixed and repeats every Davidson iteration, so
// here the planner fixes the placement once: blocks read by more than one
// term chunk or by the small-task class (and blocks read by no task) stay on
// the device, and the diagonal of H_eff reads a kept array of the diagonals
// of its blocks; the remaining device budget takes the blocks
// of the first chunks in order (the immutable data filled from the left);
// every other block is read by exactly one chunk and lies in pinned host
// memory, the blocks of a chunk contiguous, so that one cudaMemcpyAsync per
// chunk moves them into one of two device slots.  A cyclic access pattern
// larger than the buffer would evict everything under a least-recently-used
// rule; the fixed split keeps the resident fraction resident.
#include <algorithm>
#include <cstring>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "su2_device.h"

namespace su2 {

int generate_blocks(const std::vector<GenBlock>& gen, const std::vector<int>* which, double* d_arena, int64_t shift,
                    cudaStream_t s);

namespace {

struct Move {
  int64_t src, dst, n, stride;  // doubles
};

// dst[m.dst + i] = src[m.src + i * m.stride]: one CTA per (move, 64K-element piece)
__global__ void move_kernel(const Move* __restrict__ mv, const int64_t* __restrict__ piece_move,
                            const int64_t* __restrict__ piece_start, const double* __restrict__ src,
                            double* __restrict__ dst) {
  const Move m = mv[piece_move[blockIdx.x]];
  const int64_t i0 = piece_start[blockIdx.x];
  const int64_t i1 = i0 + 65536 < m.n ? i0 + 65536 : m.n;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) dst[m.dst + i] = src[m.src + i * m.stride];
}

cudaError_t run_moves(const std::vector<Move>& mv, const double* src, double* dst, cudaStream_t s) {
  if (mv.empty()) return cudaSuccess;
  std::vector<int64_t> pm, ps;
  for (size_t k = 0; k < mv.size(); ++k)
    for (int64_t i = 0; i < mv[k].n; i += 65536) {
      pm.push_back(int64_t(k));
      ps.push_back(i);
    }
  if (pm.empty()) return cudaSuccess;
  Move* dmv = nullptr;
  int64_t *dpm = nullptr, *dps = nullptr;
  cudaError_t e = cudaMalloc(&dmv, mv.size() * sizeof(Move));
  if (e == cudaSuccess) e = cudaMalloc(&dpm, pm.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&dps, ps.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMemcpy(dmv, mv.data(), mv.size() * sizeof(Move), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dpm, pm.data(), pm.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dps, ps.data(), ps.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    move_kernel<<<unsigned(pm.size()), 256, 0, s>>>(dmv, dpm, dps, src, dst);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaFree(dmv);
  cudaFree(dpm);
  cudaFree(dps);
  return e;
}

inline int64_t padded(const OpBlock& b) { return (int64_t(b.rows) * b.cols + 1) & ~int64_t(1); }

void fetch(OpStream& os, int c) {
  const int64_t n = os.he[size_t(c)] - os.hs[size_t(c)];
  if (n > 0)
    cudaMemcpyAsync(os.dbuf + os.prefix + int64_t(c & 1) * os.slot, os.host + (os.hs[size_t(c)] - os.prefix),
                    size_t(n) * sizeof(double), cudaMemcpyHostToDevice, os.io);
  cudaEventRecord(os.copied[c & 1], os.io);
}

}  // namespace

// Chunk boundaries, placement and the logical layout of an environment whose
// tasks are built; rewrites the blocks' offsets (and those of the generated
// blocks) to the logical arena and keeps the old offsets for the population.
std::string stream_plan(su2_env* env, int64_t budget, int64_t resident_bytes, std::vector<int64_t> old_off[2]) {
  OpStream& os = env->os;
  const auto& B = env->blocks;
  const auto& tasks = env->tasks;
  const int nterms = int(env->table.terms.size());
  SideOps* side[2] = {&env->L, &env->R};
  auto is_small = [&](const Task& t) {
    return std::max(std::max(B[t.f].rows, B[t.f].cols), std::max(B[t.e].rows, B[t.e].cols)) <= kSmallDim;
  };
  std::vector<std::vector<int64_t>> by_term(size_t(std::max(nterms, 1)));
  for (int64_t i = 0; i < int64_t(tasks.size()); ++i) by_term[size_t(tasks[i].term)].push_back(i);
  // chunk boundaries: the intermediates of both paths (FP64 T, float-float
  // T, T' slabs of up to six BF16 slices) and the operator blocks a chunk
  // reads each stay within the budget
  std::vector<int> starts{0};
  {
    int64_t tbytes = 0, obytes = 0;
    std::unordered_set<uint64_t> seen_t, seen_o;
    for (int ti = 0; ti < nterms; ++ti) {
      int64_t add_t = 0, add_o = 0;
      std::unordered_set<uint64_t> mine_t, mine_o;
      for (int64_t i : by_term[size_t(ti)]) {
        const Task& t = tasks[size_t(i)];
        const Block& E = B[t.e];
        const Block& F = B[t.f];
        add_t += 12 * int64_t(F.cols) * E.rows;
        if (t.dblk >= 0) {
          const uint64_t key = (uint64_t(uint32_t(t.dblk)) << 32) | uint32_t(t.e);
          if (!seen_t.count(key) && mine_t.insert(key).second) add_t += 16 * int64_t(E.rows) * env->R.blocks[t.dblk].rows;
        }
        for (int sd = 0; sd < 2; ++sd) {
          const int b = sd == 0 ? t.ablk : t.dblk;
          if (b < 0) continue;
          const uint64_t key = (uint64_t(sd) << 32) | uint32_t(b);
          if (!seen_o.count(key) && mine_o.insert(key).second) add_o += 8 * padded(side[sd]->blocks[size_t(b)]);
        }
      }
      if ((tbytes > 0 || obytes > 0) && (tbytes + add_t > budget || obytes + add_o > budget)) {
        starts.push_back(ti);
        seen_t.clear();
        seen_o.clear();
        tbytes = obytes = 0;
      }
      seen_t.insert(mine_t.begin(), mine_t.end());
      seen_o.insert(mine_o.begin(), mine_o.end());
      tbytes += add_t;
      obytes += add_o;
    }
    starts.push_back(nterms);
  }
  const int nch = int(starts.size()) - 1;
  std::vector<int> chunk_of(size_t(std::max(nterms, 1)), 0);
  for (int c = 0; c < nch; ++c)
    for (int ti = starts[size_t(c)]; ti < starts[size_t(c) + 1]; ++ti) chunk_of[size_t(ti)] = c;
  // readers of each block
  std::vector<int> first[2];
  std::vector<char> pinned[2];
  for (int sd = 0; sd < 2; ++sd) {
    first[sd].assign(side[sd]->blocks.size(), -1);
    pinned[sd].assign(side[sd]->blocks.size(), 0);
  }
  for (const Task& t : tasks) {
    const int c = chunk_of[size_t(t.term)];
    for (int sd = 0; sd < 2; ++sd) {
      const int b = sd == 0 ? t.ablk : t.dblk;
      if (b < 0) continue;
      if (is_small(t)) pinned[sd][size_t(b)] = 1;  // small-task class
      int& f = first[sd][size_t(b)];
      if (f < 0) f = c;
      else if (f != c) pinned[sd][size_t(b)] = 1;  // read by several chunks
    }
  }
  // residency: the pinned blocks and the unread ones, then the blocks of the
  // first chunks while the budget lasts
  int64_t res = 0;
  std::vector<char> resident[2];
  for (int sd = 0; sd < 2; ++sd) {
    resident[sd].assign(side[sd]->blocks.size(), 0);
    for (size_t b = 0; b < side[sd]->blocks.size(); ++b)
      if (pinned[sd][b] || first[sd][b] < 0) {
        resident[sd][b] = 1;
        res += 8 * padded(side[sd]->blocks[b]);
      }
  }
  std::vector<std::vector<std::pair<int, int>>> owned(size_t(std::max(nch, 1)));  // (side, block) read by one chunk
  for (int sd = 0; sd < 2; ++sd)
    for (size_t b = 0; b < side[sd]->blocks.size(); ++b)
      if (!resident[sd][b]) owned[size_t(first[sd][b])].push_back({sd, int(b)});
  for (int c = 0; c < nch; ++c)
    for (const auto& x : owned[size_t(c)]) {
      const int64_t sz = 8 * padded(side[x.first]->blocks[size_t(x.second)]);
      if (res + sz > resident_bytes) break;
      resident[x.first][size_t(x.second)] = 1;
      res += sz;
    }
  // logical layout: resident blocks (left, then right), then each chunk's
  // streamed blocks
  for (int sd = 0; sd < 2; ++sd) {
    old_off[sd].resize(side[sd]->blocks.size());
    for (size_t b = 0; b < side[sd]->blocks.size(); ++b) old_off[sd][b] = side[sd]->blocks[b].off;
  }
  int64_t off = 0;
  for (int sd = 0; sd < 2; ++sd)
    for (size_t b = 0; b < side[sd]->blocks.size(); ++b)
      if (resident[sd][b]) {
        side[sd]->blocks[b].off = off;
        off += padded(side[sd]->blocks[b]);
      }
  os.prefix = off;
  os.hs.assign(size_t(nch), 0);
  os.he.assign(size_t(nch), 0);
  os.slot = 0;
  for (int c = 0; c < nch; ++c) {
    os.hs[size_t(c)] = off;
    for (const auto& x : owned[size_t(c)]) {
      if (resident[x.first][size_t(x.second)]) continue;
      OpBlock& ob = side[x.first]->blocks[size_t(x.second)];
      ob.off = off;
      off += padded(ob);
    }
    os.he[size_t(c)] = off;
    os.slot = std::max(os.slot, off - os.hs[size_t(c)]);
  }
  os.total = off;
  os.io_bytes = 8.0 * double(os.total - os.prefix);
  // diagonals read by the diagonal of H_eff (tasks with e == f; their blocks are square)
  os.dg_total = 0;
  for (int sd = 0; sd < 2; ++sd) os.dg_off[sd].assign(side[sd]->blocks.size(), -1);
  for (const Task& t : tasks) {
    if (t.e != t.f) continue;
    for (int sd = 0; sd < 2; ++sd) {
      const int b = sd == 0 ? t.ablk : t.dblk;
      if (b < 0 || os.dg_off[sd][size_t(b)] >= 0) continue;
      os.dg_off[sd][size_t(b)] = os.dg_total;
      os.dg_total += side[sd]->blocks[size_t(b)].rows;
    }
  }
  os.starts = starts;
  // generated blocks follow their blocks
  for (int sd = 0; sd < 2; ++sd) {
    if (side[sd]->gen.empty()) continue;
    std::unordered_map<int64_t, int64_t> moved;
    for (size_t b = 0; b < side[sd]->blocks.size(); ++b) moved[old_off[sd][b]] = side[sd]->blocks[b].off;
    for (GenBlock& g : side[sd]->gen) g.off = moved.at(g.off);
  }
  os.on = true;
  return "";
}

// Device buffer, pinned host arena, IO stream and events; fills the resident
// part and the host arena from the operator source of each side: generated
// entries, a host arena, or a device arena the builder left (dev_old, freed
// by the caller).
std::string stream_populate(su2_env* env, cudaStream_t s, double* dev_old[2], const std::vector<int64_t> old_off[2]) {
  OpStream& os = env->os;
  SideOps* side[2] = {&env->L, &env->R};
  const int nch = int(os.starts.size()) - 1;
  auto cu = [](cudaError_t e, const char* what) -> std::string {
    return e == cudaSuccess ? "" : std::string("out-of-core operators: ") + what + ": " + cudaGetErrorString(e);
  };
  std::string err;
  const int64_t dn = std::max<int64_t>(os.prefix + 2 * os.slot, 2);
  if (cudaMalloc(&os.dbuf, size_t(dn) * sizeof(double)) != cudaSuccess) {
    (void)cudaGetLastError();
    os.dbuf = nullptr;
    return "out-of-core operators: device allocation of the resident part and the slots failed";
  }
  const int64_t hn = std::max<int64_t>(os.total - os.prefix, 2);
  if (cudaHostAlloc((void**)&os.host, size_t(hn) * sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
    (void)cudaGetLastError();
    os.host = nullptr;
    return "out-of-core operators: pinned host allocation failed";
  }
  err = cu(cudaStreamCreateWithFlags(&os.io, cudaStreamNonBlocking), "IO stream");
  for (int k = 0; k < 2 && err.empty(); ++k) {
    err = cu(cudaEventCreateWithFlags(&os.copied[k], cudaEventDisableTiming), "events");
    if (err.empty()) err = cu(cudaEventCreateWithFlags(&os.freed[k], cudaEventDisableTiming), "events");
  }
  if (err.empty()) err = cu(cudaEventCreateWithFlags(&os.fork, cudaEventDisableTiming), "events");
  if (err.empty()) err = cu(cudaEventCreateWithFlags(&os.join, cudaEventDisableTiming), "events");
  if (!err.empty()) return err;
  // the range [lo, hi) of the logical arena written at dst + (off - lo)
  if (cudaMalloc(&os.ddiag, size_t(std::max<int64_t>(os.dg_total, 2)) * sizeof(double)) != cudaSuccess) {
    (void)cudaGetLastError();
    os.ddiag = nullptr;
    return "out-of-core operators: device allocation of the diagonals failed";
  }
  // the range [lo, hi) of the logical arena written at dst + (off - lo);
  // the diagonals the diagonal of H_eff reads are taken from there
  auto fill = [&](int64_t lo, int64_t hi, double* dst) -> std::string {
    std::vector<Move> dg;
    for (int sd = 0; sd < 2; ++sd) {
      SideOps& so = *side[sd];
      std::vector<int> which;
      std::vector<Move> mv;
      for (size_t b = 0; b < so.blocks.size(); ++b) {
        const OpBlock& ob = so.blocks[b];
        if (ob.off < lo || ob.off >= hi) continue;
        const int64_t n = int64_t(ob.rows) * ob.cols;
        if (os.dg_off[sd][b] >= 0) dg.push_back(Move{ob.off - lo, os.dg_off[sd][b], ob.rows, ob.rows + 1});
        if (dev_old[sd]) {
          mv.push_back(Move{old_off[sd][b], ob.off - lo, n, 1});
        } else if (so.host_values) {
          if (n > 0) {
            const cudaError_t e = cudaMemcpy(dst + (ob.off - lo), &so.arena[size_t(old_off[sd][b])],
                                             size_t(n) * sizeof(double), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cu(e, "upload");
          }
        }
      }
      if (dev_old[sd]) {
        std::string e = cu(run_moves(mv, dev_old[sd], dst, s), "gather");
        if (!e.empty()) return e;
      } else if (!so.host_values) {
        for (size_t g = 0; g < so.gen.size(); ++g)
          if (so.gen[g].off >= lo && so.gen[g].off < hi) which.push_back(int(g));
        const int ce = generate_blocks(so.gen, &which, dst, lo, s);
        if (ce) return cu(cudaError_t(ce), "generation");
      }
    }
    return cu(run_moves(dg, dst, os.ddiag, s), "diagonals");
  };
  err = fill(0, os.prefix, os.dbuf);
  for (int c = 0; c < nch && err.empty(); ++c) {
    const int64_t lo = os.hs[size_t(c)], hi = os.he[size_t(c)];
    if (hi == lo) continue;
    double* stage = os.dbuf + os.prefix;
    err = fill(lo, hi, stage);
    if (err.empty())
      err = cu(cudaMemcpy(os.host + (lo - os.prefix), stage, size_t(hi - lo) * sizeof(double), cudaMemcpyDeviceToHost),
               "download");
  }
  if (err.empty()) err = cu(cudaStreamSynchronize(s), "population");
  if (err.empty())
    for (int sd = 0; sd < 2; ++sd) {  // the host copies are no longer the layout of the blocks
      side[sd]->arena.clear();
      side[sd]->arena.shrink_to_fit();
      side[sd]->host_values = false;
      side[sd]->gen.clear();
    }
  return err;
}

void stream_free(OpStream& os) {
  if (os.io) cudaStreamSynchronize(os.io);
  cudaFree(os.dbuf);
  cudaFree(os.ddiag);
  cudaFreeHost(os.host);
  for (int k = 0; k < 2; ++k) {
    if (os.copied[k]) cudaEventDestroy(os.copied[k]);
    if (os.freed[k]) cudaEventDestroy(os.freed[k]);
  }
  if (os.fork) cudaEventDestroy(os.fork);
  if (os.join) cudaEventDestroy(os.join);
  if (os.io) cudaStreamDestroy(os.io);
  os = OpStream();
}

// One H.psi over the chunks: begin (the IO stream follows the compute stream
// and copies chunks 0 and 1), then per chunk c wait (the compute stream waits
// for chunk c's copy) and release (after chunk c's last reader of its slot:
// the copy of chunk c + 2 into the same slot), then end (the compute stream
// waits for the IO stream).
void stream_begin(OpStream& os, cudaStream_t s) {
  cudaEventRecord(os.fork, s);
  cudaStreamWaitEvent(os.io, os.fork, 0);
  const int nch = int(os.starts.size()) - 1;
  for (int c = 0; c < std::min(2, nch); ++c) fetch(os, c);
}
void stream_wait(OpStream& os, int c, cudaStream_t s) { cudaStreamWaitEvent(s, os.copied[c & 1], 0); }
void stream_release(OpStream& os, int c, cudaStream_t s) {
  const int nch = int(os.starts.size()) - 1;
  cudaEventRecord(os.freed[c & 1], s);
  if (c + 2 < nch) {
    cudaStreamWaitEvent(os.io, os.freed[c & 1], 0);
    fetch(os, c + 2);
  }
}
void stream_end(OpStream& os, cudaStream_t s) {
  cudaEventRecord(os.join, os.io);
  cudaStreamWaitEvent(s, os.join, 0);
}

}  // namespace su2
