// C-ABI of su2dmrg (include/su2dmrg.h): contexts, sector-table, environment
// with its execution plan, H.psi, the H_eff diagonal and the Davidson driver.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <chrono>
#include <unordered_map>

#include "su2_device.h"

namespace su2 {
int dav_grid(int64_t n);
void dav_multidot(cudaStream_t, const double*, int64_t, int, const double*, int64_t, double*, double*, double,
                  const int* dn = nullptr);
void dav_combine(cudaStream_t, const double*, const double*, int64_t, int, const double*, int64_t, double*, double*,
                 const int* dn = nullptr);
void dav_subtract(cudaStream_t, const double*, int64_t, int, const double*, int64_t, double*, const int* dn = nullptr);
void dav_residual(cudaStream_t, const double*, const double*, const double*, int64_t, double*);
void dav_precond(cudaStream_t, const double*, const double*, const double*, int64_t, double*);
void dav_scale(cudaStream_t, double*, const double*, const double*, int64_t);
void dav_jacobi(cudaStream_t, const double*, int, int, double*, double*, int*, const int* dn = nullptr);
void dav_absmax(cudaStream_t, const double*, int64_t, double*, int64_t*, int*);
void dav_diag_set(cudaStream_t, double*, int, int, const double*);
void dav_copy_col(cudaStream_t, double*, int, int, const double*, int, const int* dn = nullptr);
void dav_newest(cudaStream_t, double*, int64_t, const int*, double*, int);
void dav_restart(cudaStream_t, double*, double*, int64_t, const double*, int, double*, const double*, int, int, int*,
                 double*);
void dav_append(cudaStream_t, double*, int64_t, int*, const double*, const double*);
// split-precision path (heff_split.cu)
int split_prepare(su2_env* env, int n_slices, std::string& err);
int split_autotune(su2_env* env, double tol, std::string& err);
int generate_side(const SideOps& so, double* d_arena, cudaStream_t s);
int split_apply(su2_env* env, const double* psi, double* F, std::string& err);
std::string stream_plan(su2_env* env, int64_t budget, int64_t resident_bytes, std::vector<int64_t> old_off[2]);
std::string stream_populate(su2_env* env, cudaStream_t s, double* dev_old[2], const std::vector<int64_t> old_off[2]);
void stream_free(OpStream& os);
void stream_begin(OpStream& os, cudaStream_t s);
void stream_wait(OpStream& os, int c, cudaStream_t s);
void stream_release(OpStream& os, int c, cudaStream_t s);
void stream_end(OpStream& os, cudaStream_t s);
void split_free(su2_env* env);
}  // namespace su2

using namespace su2;

namespace {

int fail(su2_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

#define CUDA_TRY(ctx, call)                                                               \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(ctx, SU2_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool fail_alloc_injected() {
  const char* s = std::getenv("SU2_FAIL_ALLOC");
  return s && s[0] == '1';
}

template <class T>
int dev_alloc(su2_ctx* ctx, T** p, size_t count) {
  *p = nullptr;
  if (fail_alloc_injected()) return fail(ctx, SU2_ENOMEM, "device allocation refused (SU2_FAIL_ALLOC=1)");
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(ctx, SU2_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return SU2_OK;
}

template <class T>
int upload(su2_ctx* ctx, T** d, const std::vector<T>& h) {
  int rc = dev_alloc(ctx, d, h.size());
  if (rc) return rc;
  if (!h.empty()) CUDA_TRY(ctx, cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SU2_OK;
}

int set_device(su2_ctx* ctx) {
  if (ctx->device < 0) return fail(ctx, SU2_EINVAL, "host-only context cannot run device work");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  // an error latched in this thread by code outside the library (it is
  // reported to whoever made that call) must not fail the launch checks below
  (void)cudaGetLastError();
  return SU2_OK;
}

// Reads and clears the device status word; call after the context stream has
// been synchronised.  A non-zero word (a bounded device wait gave up) turns
// into SU2_ETIMEOUT, so a call that synchronises never reports success for a
// result computed by a kernel that aborted.
int device_status_rc(su2_ctx* ctx) {
  int v = 0;
  CUDA_TRY(ctx, cudaMemcpy(&v, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (v == 0) return SU2_OK;
  CUDA_TRY(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
  return fail(ctx, SU2_ETIMEOUT, "a bounded device-side wait gave up (device status " + std::to_string(v) + ")");
}

}  // namespace

extern "C" {

int su2_ctx_create(int device, void* cuda_stream, su2_ctx** out) {
  if (!out) return SU2_EINVAL;
  *out = nullptr;
  su2_ctx* c = new (std::nothrow) su2_ctx();
  if (!c) return SU2_ENOMEM;
  c->device = device;
  if (device >= 0) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device >= n) {
      delete c;
      return SU2_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
      delete c;
      return SU2_ECUDA;
    }
    c->stream = (cudaStream_t)cuda_stream;  // NULL: the legacy default stream
    if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess || cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess) {
      delete c;
      return SU2_ECUDA;
    }
  }
  *out = c;
  return SU2_OK;
}

int su2_ctx_destroy(su2_ctx* ctx) {
  if (!ctx) return SU2_EINVAL;
  if (ctx->device >= 0) {
    cudaSetDevice(ctx->device);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  }
  delete ctx;
  return SU2_OK;
}

const char* su2_last_error(su2_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int su2_ctx_wait(su2_ctx* ctx, double timeout_s) {
  if (!ctx) return SU2_EINVAL;
  int rc = set_device(ctx);
  if (rc) return rc;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(ctx->stream);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return fail(ctx, SU2_ECUDA, std::string("cudaStreamQuery: ") + cudaGetErrorString(e));
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_s >= 0.0 && dt > timeout_s)
      return fail(ctx, SU2_ETIMEOUT, "host watchdog: the context stream is still busy after the time limit");
    std::this_thread::sleep_for(std::chrono::microseconds(dt < 1e-3 ? 10 : 200));
  }
  return device_status_rc(ctx);
}

int su2_ctx_status(su2_ctx* ctx, int32_t* device_status) {
  if (!ctx || !device_status) return fail(ctx, SU2_EINVAL, "null argument");
  int rc = set_device(ctx);
  if (rc) return rc;
  int v = 0;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  CUDA_TRY(ctx, cudaMemcpy(&v, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
  *device_status = v;
  return SU2_OK;
}

int su2_build_sectors(su2_ctx* ctx, const su2_sector* left, int32_t n_left, const su2_sector* right, int32_t n_right,
                      int32_t site_kind, int32_t N_target, int32_t twoS_target, su2_sectors** out) {
  if (!ctx || !out || (!left && n_left) || (!right && n_right) || n_left < 0 || n_right < 0)
    return fail(ctx, SU2_EINVAL, "null argument");
  *out = nullptr;
  if (site_kind != SU2_SITE_SPIN_HALF && site_kind != SU2_SITE_ORBITAL) return fail(ctx, SU2_EINVAL, "site_kind");
  if (twoS_target < 0 || N_target < 0) return fail(ctx, SU2_EINVAL, "negative target");
  su2_sectors* s = new (std::nothrow) su2_sectors();
  if (!s) return fail(ctx, SU2_ENOMEM, "host allocation");
  s->site_kind = site_kind;
  s->N = N_target;
  s->twoS = twoS_target;
  auto check = [&](const su2_sector* v, int n, std::vector<Sector>& dst) {
    for (int i = 0; i < n; ++i) {
      if (v[i].dim < 1 || v[i].twoS < 0 || v[i].N < 0 || ((v[i].N - v[i].twoS) % 2 != 0 && site_kind == SU2_SITE_ORBITAL))
        return false;
      if (i > 0 && !(v[i - 1].N < v[i].N || (v[i - 1].N == v[i].N && v[i - 1].twoS < v[i].twoS))) return false;
      dst.push_back(Sector{v[i].N, v[i].twoS, v[i].dim});
    }
    return true;
  };
  if (!check(left, n_left, s->left) || !check(right, n_right, s->right)) {
    delete s;
    return fail(ctx, SU2_EINVAL, "sectors must have dim >= 1, valid (N, 2S) and ascending order");
  }
  build_blocks(s->left, s->right, site_kind, N_target, twoS_target, s->blocks, s->psi_len);
  for (const Block& b : s->blocks) s->pub.push_back(su2_block{b.a, b.s1, b.s2, b.b, b.jL1, b.j2R, b.rows, b.cols, b.offset});
  *out = s;
  return SU2_OK;
}

int su2_sectors_query(const su2_sectors* s, int64_t* psi_len, int32_t* n_blocks, const su2_block** blocks) {
  if (!s) return SU2_EINVAL;
  if (psi_len) *psi_len = s->psi_len;
  if (n_blocks) *n_blocks = int32_t(s->blocks.size());
  if (blocks) *blocks = s->pub.data();
  return SU2_OK;
}

int su2_sectors_destroy(su2_sectors* s) {
  if (!s) return SU2_EINVAL;
  delete s;
  return SU2_OK;
}

static int build_plan(su2_env* env, const su2_sectors* S, int64_t budget) {
  const auto& tasks = env->tasks;
  const auto& blocks = S->blocks;
  const int nterms = int(env->table.terms.size());
  // uniques of K1 per term (first appearance order)
  std::vector<std::vector<int64_t>> by_term(nterms);
  for (int64_t i = 0; i < int64_t(tasks.size()); ++i) by_term[tasks[i].term].push_back(i);
  // chunk boundaries over terms (out-of-core: the planner's)
  std::vector<int> starts;
  if (env->os.on) {
    starts = env->os.starts;
  } else {
    std::unordered_map<uint64_t, int64_t> seen;
    int64_t bytes = 0;
    starts.push_back(0);
    for (int ti = 0; ti < nterms; ++ti) {
      int64_t add = 0;
      std::unordered_map<uint64_t, int64_t> mine;
      for (int64_t i : by_term[ti]) {
        const Task& t = tasks[i];
        if (t.dblk < 0) continue;
        const uint64_t key = (uint64_t(uint32_t(t.dblk)) << 32) | uint32_t(t.e);
        if (seen.count(key) || mine.count(key)) continue;
        const int64_t sz = int64_t(blocks[t.e].rows) * env->R.blocks[t.dblk].rows * 8;
        mine[key] = sz;
        add += sz;
      }
      if (bytes > 0 && bytes + add > budget) {
        starts.push_back(ti);
        seen.clear();
        bytes = 0;
      }
      for (auto& kv : mine) seen.insert(kv);
      bytes += add;
    }
    starts.push_back(nterms);
  }
  double flops = 0.0;
  int64_t max_t = 0, nk1 = 0;
  for (size_t c = 0; c + 1 < starts.size(); ++c) {
    const int t0 = starts[c], t1 = starts[c + 1];
    Chunk ch{int64_t(env->k1.size()), 0, int64_t(env->k2.size()), 0, 0.0, 0.0};
    std::unordered_map<uint64_t, int64_t> toff;  // key -> offset in T buffer
    int64_t tsz = 0;
    // K1 uniques in term order
    for (int ti = t0; ti < t1; ++ti)
      for (int64_t i : by_term[ti]) {
        const Task& t = tasks[i];
        if (t.dblk < 0) continue;
        const uint64_t key = (uint64_t(uint32_t(t.dblk)) << 32) | uint32_t(t.e);
        if (toff.count(key)) continue;
        const Block& E = blocks[t.e];
        const OpBlock& D = env->R.blocks[t.dblk];
        toff[key] = tsz;
        const int k1 = E.rows, k2 = E.cols, n = D.rows;
        for (int tc = 0; tc < (n + kTile - 1) / kTile; ++tc)
          for (int tr = 0; tr < (k1 + kTile - 1) / kTile; ++tr)
            env->k1.push_back(K1Job{E.offset, env->os.on ? env->os.dev_off(D.off, int(c)) : D.off, tsz, k1, k2, n,
                                    tr, tc, 0});
        flops += 2.0 * k1 * k2 * n;
        ch.k1_flops += 2.0 * k1 * k2 * n;
        ++nk1;
        tsz += (int64_t(k1) * n + 1) & ~int64_t(1);
      }
    max_t = std::max(max_t, tsz);
    ch.k1_end = int64_t(env->k1.size());
    // K2: tasks of the chunk in (f, term, e) order, grouped by f
    std::vector<K2Job> jobs;
    std::vector<double> cost;
    int64_t i = 0;
    const int64_t nt = int64_t(tasks.size());
    while (i < nt) {
      const int f = tasks[i].f;
      int64_t j = i;
      const int64_t tb = int64_t(env->k2t.size());
      double c2 = 0.0;
      for (; j < nt && tasks[j].f == f; ++j) {
        const Task& t = tasks[j];
        if (t.term < t0 || t.term >= t1) continue;
        const Block& E = blocks[t.e];
        const Block& F = blocks[t.f];
        K2Task k;
        k.k1 = E.rows;
        k.v = t.v;
        k.flags = 0;
        if (t.ablk < 0) {
          k.flags |= K2_A_IDENTITY;
          k.a_off = -1;
          c2 += 1.0;
        } else {
          k.a_off = env->os.on ? env->os.dev_off(env->L.blocks[t.ablk].off, int(c)) : env->L.blocks[t.ablk].off;
          flops += 2.0 * F.rows * E.rows * F.cols;
          ch.k2_flops += 2.0 * F.rows * E.rows * F.cols;
          c2 += E.rows;
        }
        if (t.dblk < 0) {
          k.flags |= K2_B_FROM_PSI;
          k.b_off = E.offset;
        } else {
          k.b_off = toff.at((uint64_t(uint32_t(t.dblk)) << 32) | uint32_t(t.e));
        }
        env->k2t.push_back(k);
      }
      const int64_t te = int64_t(env->k2t.size());
      if (te > tb) {
        const Block& F = blocks[f];
        for (int tc = 0; tc < (F.cols + kTile - 1) / kTile; ++tc)
          for (int tr = 0; tr < (F.rows + kTile - 1) / kTile; ++tr) {
            jobs.push_back(K2Job{F.offset, F.rows, F.cols, tr, tc, int32_t(tb), int32_t(te)});
            cost.push_back(c2);
          }
      }
      i = j;
    }
    std::vector<int64_t> ord(jobs.size());
    for (size_t q = 0; q < ord.size(); ++q) ord[q] = int64_t(q);
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
    for (int64_t q : ord) env->k2.push_back(jobs[q]);
    ch.k2_end = int64_t(env->k2.size());
    env->chunks.push_back(ch);
  }
  if (int64_t(env->k2t.size()) >= (int64_t(1) << 31)) return fail(env->ctx, SU2_EINVAL, "task table too large");
  env->t_elems = max_t;
  env->info.t_chunk_bytes = max_t * int64_t(sizeof(double));
  env->info.flops_su2 = flops;
  env->info.n_k1 = nk1;
  env->info.n_chunks = int64_t(env->chunks.size());
  // diagonal: tasks with e == f, grouped by f
  int64_t i = 0;
  const int64_t nt = int64_t(tasks.size());
  while (i < nt) {
    const int f = tasks[i].f;
    const int64_t tb = int64_t(env->dt.size());
    for (; i < nt && tasks[i].f == f; ++i) {
      const Task& t = tasks[i];
      if (t.e != t.f) continue;
      DiagTask d;
      if (env->os.on) {  // out-of-core: the kept diagonals, stride 1
        d.a_off = t.ablk < 0 ? -1 : env->os.dg_off[0][size_t(t.ablk)];
        d.d_off = t.dblk < 0 ? -1 : env->os.dg_off[1][size_t(t.dblk)];
        d.lda = d.ldd = 0;
      } else {
        d.a_off = t.ablk < 0 ? -1 : env->L.blocks[t.ablk].off;
        d.d_off = t.dblk < 0 ? -1 : env->R.blocks[t.dblk].off;
        d.lda = blocks[f].rows;
        d.ldd = blocks[f].cols;
      }
      d.v = t.v;
      env->dt.push_back(d);
    }
    const int64_t te = int64_t(env->dt.size());
    if (te > tb) env->dj.push_back(DiagJob{blocks[f].offset, blocks[f].rows, blocks[f].cols, int32_t(tb), int32_t(te)});
  }
  return SU2_OK;
}

static void env_free_device(su2_env* e) {
  if (e->device < 0) return;
  cudaSetDevice(e->device);
  split_free(e);
  if (e->os.on) {  // dL and dR point into the out-of-core buffer
    stream_free(e->os);
    e->dL = e->dR = nullptr;
  }
  cudaFree(e->dL);
  cudaFree(e->dR);
  cudaFree(e->dT);
  cudaFree(e->dk1);
  cudaFree(e->dk2);
  cudaFree(e->dk2t);
  cudaFree(e->ddj);
  cudaFree(e->ddt);
  cudaFree(e->d_in_scratch);
  cudaFree(e->d_out_scratch);
}

// Term sharding: terms go to shards by longest-processing-time order of
// their task flops (2(m k1 k2 + m k2 n) per task; ties by term index, then by
// the lower shard), and shard `rank` keeps the tasks of its terms.  The
// shards' H.psi sum to the full H.psi.
void shard_terms(std::vector<Task>& tasks, const std::vector<Block>& blocks, int nterms, int rank, int count) {
  std::vector<double> cost(size_t(nterms), 0.0);
  for (const Task& t : tasks) {
    const Block& F = blocks[t.f];
    const Block& E = blocks[t.e];
    cost[t.term] += 2.0 * (double(F.rows) * E.rows * E.cols + double(F.rows) * E.cols * F.cols);
  }
  std::vector<int> order(static_cast<size_t>(nterms));
  for (int i = 0; i < nterms; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> load(size_t(count), 0.0);
  std::vector<int> owner(size_t(nterms), 0);
  for (int term : order) {
    int best = 0;
    for (int r = 1; r < count; ++r)
      if (load[r] < load[best]) best = r;
    owner[term] = best;
    load[best] += cost[term];
  }
  std::vector<Task> kept;
  for (const Task& t : tasks)
    if (owner[t.term] == rank) kept.push_back(t);
  tasks.swap(kept);
}

}  // extern "C"

// Execution plan, environment info, device uploads and the split-precision
// arenas of an environment whose table, operators and tasks are set; on
// failure the environment is deleted.
static int finish_env(su2_ctx* ctx, su2_env* env, const su2_sectors* S, const su2_env_opts* opts) {
  int64_t budget = (opts && opts->t_budget_bytes > 0) ? opts->t_budget_bytes : (int64_t(2) << 30);
  std::vector<int64_t> old_off[2];
  if (opts && opts->resident_bytes > 0) {
    // chunk budget: a quarter of the device memory left beside the resident
    // part, at most 16 GiB (the resident path's rule), 4 GiB on a host context
    int64_t sb = int64_t(4) << 30;
    if (opts->t_budget_bytes > 0) {
      sb = opts->t_budget_bytes;
    } else if (ctx->device >= 0) {
      size_t fr = 0, tot = 0;
      if (set_device(ctx) == SU2_OK && cudaMemGetInfo(&fr, &tot) == cudaSuccess)
        sb = std::min<int64_t>(int64_t(16) << 30,
                               std::max<int64_t>((int64_t(fr) - opts->resident_bytes) / 4, int64_t(1) << 30));
    }
    std::string err = stream_plan(env, sb, opts->resident_bytes, old_off);
    if (!err.empty()) {
      cudaFree(env->L.dev_ready);
      cudaFree(env->R.dev_ready);
      delete env;
      return fail(ctx, SU2_EINVAL, err);
    }
    env->split_budget = sb;
    if (ctx->device < 0) {
      // host context: the plan only (its numbers in the info); each side's
      // host arena takes the logical layout
      for (int sd = 0; sd < 2; ++sd) {
        SideOps& so = sd == 0 ? env->L : env->R;
        std::vector<double> a(size_t(std::max<int64_t>(env->os.total, 2)), 0.0);
        for (size_t b = 0; b < so.blocks.size(); ++b)
          std::memcpy(&a[size_t(so.blocks[b].off)], &so.arena[size_t(old_off[sd][b])],
                      sizeof(double) * size_t(so.blocks[b].rows) * so.blocks[b].cols);
        so.arena.swap(a);
      }
    }
  }
  int rc2 = build_plan(env, S, budget);
  if (rc2) {
    delete env;
    return rc2;
  }
  // info
  su2_env_info& in = env->info;
  in.psi_len = S->psi_len;
  in.n_blocks = int64_t(S->blocks.size());
  in.n_terms = int64_t(env->table.terms.size());
  in.n_tasks = int64_t(env->tasks.size());
  double D = 0, Deff = 0;
  for (const Sector& s : S->left) {
    D += s.dim;
    Deff += double(s.dim) * (s.twoS + 1);
  }
  in.r_d = D > 0 ? Deff / D : 1.0;
  in.flops_u1_equiv = in.flops_su2 * in.r_d;
  {
    // the same U(1) counting with the tasks of all shards (a shard's own count
    // would need the expansion of its own terms only; counted on the full table)
    in.flops_u1_counted = u1_counted_flops(env->table, S->left, S->right, S->N, S->twoS);
    in.r_cc = in.flops_su2 > 0 ? in.flops_u1_counted / in.flops_su2 : 0.0;
  }
  in.env_bytes = 8.0 * double(env->L.arena_size + env->R.arena_size);
  in.resident_bytes = env->os.on ? 8 * env->os.prefix : int64_t(in.env_bytes);
  in.streamed_bytes = env->os.on ? 8 * (env->os.total - env->os.prefix) : 0;
  in.n_io_chunks = env->os.on ? int64_t(env->os.starts.size()) - 1 : 0;
  if (ctx->device >= 0 && env->os.on) {
    int rc = set_device(ctx);
    if (!rc) {
      double* dev_old[2] = {env->L.dev_ready, env->R.dev_ready};
      const std::string err = stream_populate(env, ctx->stream, dev_old, old_off);
      cudaFree(dev_old[0]);
      cudaFree(dev_old[1]);
      env->L.dev_ready = env->R.dev_ready = nullptr;
      env->dL = env->dR = env->os.dbuf;
      if (!err.empty()) rc = fail(ctx, SU2_ENOMEM, err);
    }
    if (rc) {
      env_free_device(env);
      delete env;
      return rc;
    }
  }
  if (ctx->device >= 0) {
    int rc = set_device(ctx);
    for (int side = 0; side < 2 && !rc && !env->os.on; ++side) {
      SideOps& so = side == 0 ? env->L : env->R;
      double** dst = side == 0 ? &env->dL : &env->dR;
      if (so.dev_ready) {  // filled on the device by the builder
        *dst = so.dev_ready;
        so.dev_ready = nullptr;
      } else if (so.host_values) {
        rc = upload(ctx, dst, so.arena);
      } else {
        rc = dev_alloc(ctx, dst, size_t(std::max<int64_t>(so.arena_size, 2)));
        if (!rc) {
          const int ce = generate_side(so, *dst, ctx->stream);
          if (ce) rc = fail(ctx, SU2_ECUDA, std::string("operator generation: ") + cudaGetErrorString(cudaError_t(ce)));
        }
      }
    }
    if (!rc) rc = dev_alloc(ctx, &env->dT, size_t(std::max<int64_t>(env->t_elems, 2)));
    if (!rc) rc = upload(ctx, &env->dk1, env->k1);
    if (!rc) rc = upload(ctx, &env->dk2, env->k2);
    if (!rc) rc = upload(ctx, &env->dk2t, env->k2t);
    if (!rc) rc = upload(ctx, &env->ddj, env->dj);
    if (!rc) rc = upload(ctx, &env->ddt, env->dt);
    if (!rc && opts && (opts->prepare_split || opts->autotune)) {
      std::string err;
      if (opts->autotune) rc = split_autotune(env, opts->split_tol > 0 ? opts->split_tol : 3e-11, err);
      else rc = split_prepare(env, opts->n_slices > 0 ? opts->n_slices : 5, err);
      if (rc) fail(ctx, rc, err);
    }
    if (rc) {
      env_free_device(env);
      delete env;
      return rc;
    }
  }
  return SU2_OK;
}


extern "C" {

int su2_build_environment(su2_ctx* ctx, const su2_hamiltonian* H, const su2_bond_chain* lc, const su2_bond_chain* rc,
                          const su2_sectors* S, const su2_env_opts* opts, su2_env** out) {
  if (!ctx || !H || !lc || !rc || !S || !out) return fail(ctx, SU2_EINVAL, "null argument");
  *out = nullptr;
  if (H->model < 0 || H->model > 4) return fail(ctx, SU2_EINVAL, "unknown model");
  if (((H->model == SU2_MODEL_HEISENBERG) != (S->site_kind == SU2_SITE_SPIN_HALF) && H->model <= 1) ||
      (H->model == SU2_MODEL_AB_INITIO && S->site_kind != SU2_SITE_ORBITAL))
    return fail(ctx, SU2_EINVAL, "model and site kind disagree");
  if (H->model == SU2_MODEL_QC_SKELETON && (H->n_left < 1 || H->n_right < 1))
    return fail(ctx, SU2_EINVAL, "n_left and n_right must be >= 1");
  auto chain_of = [&](const su2_bond_chain* c, std::vector<std::vector<Sector>>& dst) {
    if (c->n_bonds < 1 || !c->bond_offset || !c->sectors) return false;
    for (int k = 0; k < c->n_bonds; ++k) {
      std::vector<Sector> v;
      for (int i = c->bond_offset[k]; i < c->bond_offset[k + 1]; ++i)
        v.push_back(Sector{c->sectors[i].N, c->sectors[i].twoS, c->sectors[i].dim});
      dst.push_back(v);
    }
    return true;
  };
  std::vector<std::vector<Sector>> lch, rch;
  if (!chain_of(lc, lch) || !chain_of(rc, rch)) return fail(ctx, SU2_EINVAL, "bad bond chain");
  auto same = [](const std::vector<Sector>& a, const std::vector<Sector>& b) {
    if (a.size() != b.size()) return false;
    for (size_t i = 0; i < a.size(); ++i)
      if (a[i].N != b[i].N || a[i].twoS != b[i].twoS || a[i].dim != b[i].dim) return false;
    return true;
  };
  if (!same(lch.back(), S->left) || !same(rch.back(), S->right))
    return fail(ctx, SU2_EINVAL, "last bond of a chain differs from the sector lists");
  su2_env* env = new (std::nothrow) su2_env();
  if (!env) return fail(ctx, SU2_ENOMEM, "host allocation");
  env->ctx = ctx;
  env->device = ctx->device;
  env->psi_len = S->psi_len;
  env->blocks = S->blocks;
  env->lsec = S->left;
  env->rsec = S->right;
  env->split_budget = (opts && opts->t_budget_bytes > 0) ? opts->t_budget_bytes : 0;
  env->spin_limit = (opts && opts->spin_limit > 0) ? opts->spin_limit : 0;
  try {
    std::string err;
    if (H->model == SU2_MODEL_AB_INITIO) {
      if (ctx->device >= 0 && cudaSetDevice(ctx->device) != cudaSuccess) err = "cudaSetDevice failed";
      if (err.empty())
        err = build_abinitio(*H, lch, rch, ctx->device, ctx->stream, env->split_budget, env->table, env->L, env->R,
                             &env->info.renorm_flops);
    } else {
      env->table = make_table(*H, S->site_kind);
      const bool host_values = ctx->device < 0;
      err = build_side_ops(env->table, true, lch, *H, env->L, host_values);
      if (err.empty()) err = build_side_ops(env->table, false, rch, *H, env->R, host_values);
    }
    if (err.empty()) err = build_tasks(env->table, S->left, S->right, S->blocks, S->twoS, env->L, env->R, env->tasks);
    if (err.empty() && opts && opts->shard_count > 1) {
      if (opts->shard_rank < 0 || opts->shard_rank >= opts->shard_count) err = "shard_rank outside [0, shard_count)";
      else shard_terms(env->tasks, S->blocks, int(env->table.terms.size()), opts->shard_rank, opts->shard_count);
    }
    if (!err.empty()) {
      delete env;
      return fail(ctx, SU2_EINVAL, err);
    }
  } catch (const std::bad_alloc&) {
    delete env;
    return fail(ctx, SU2_ENOMEM, "host allocation");
  } catch (const std::exception& ex) {
    delete env;
    return fail(ctx, SU2_EINVAL, ex.what());
  }
  {
    const int rcf = finish_env(ctx, env, S, opts);
    if (rcf) return rcf;
  }
  *out = env;
  return SU2_OK;
}

int su2_env_query(const su2_env* env, su2_env_info* info) {
  if (!env || !info) return SU2_EINVAL;
  *info = env->info;
  return SU2_OK;
}

int su2_env_tasks(const su2_env* env, int32_t* rows8, double* v, int64_t n_tasks) {
  if (!env || n_tasks != int64_t(env->tasks.size())) return SU2_EINVAL;
  for (int64_t i = 0; i < n_tasks; ++i) {
    const Task& t = env->tasks[i];
    if (rows8) {
      int32_t* r = rows8 + 8 * i;
      r[0] = t.f; r[1] = t.term; r[2] = t.e; r[3] = t.ao; r[4] = t.ai; r[5] = t.bo; r[6] = t.bi;
      r[7] = (t.ablk < 0 ? 1 : 0) | (t.dblk < 0 ? 2 : 0);
    }
    if (v) v[i] = t.v;
  }
  return SU2_OK;
}

int su2_env_terms(const su2_env* env, int32_t* a_op, int32_t* d_op, int32_t* k, double* alpha, int64_t n_terms) {
  if (!env || n_terms != int64_t(env->table.terms.size())) return SU2_EINVAL;
  for (int64_t i = 0; i < n_terms; ++i) {
    const Term& t = env->table.terms[size_t(i)];
    if (a_op) a_op[i] = t.A;
    if (d_op) d_op[i] = t.D;
    if (k) k[i] = t.k;
    if (alpha) alpha[i] = t.alpha;
  }
  return SU2_OK;
}

int su2_env_operator_block(const su2_env* env, int32_t side, int32_t op, int32_t qo, int32_t qi, double* out,
                           int32_t rows, int32_t cols) {
  if (!env || !out || (side != 0 && side != 1)) return SU2_EINVAL;
  const SideOps& so = side == 0 ? env->L : env->R;
  const int b = so.find(op, qo, qi);
  if (b < 0 || so.blocks[b].rows != rows || so.blocks[b].cols != cols) return SU2_EINVAL;
  if (so.host_values) {
    std::memcpy(out, &so.arena[so.blocks[b].off], sizeof(double) * size_t(rows) * cols);
    return SU2_OK;
  }
  if (env->os.on && so.blocks[b].off >= env->os.prefix) {  // out-of-core: in pinned host memory
    std::memcpy(out, env->os.host + (so.blocks[b].off - env->os.prefix), sizeof(double) * size_t(rows) * cols);
    return SU2_OK;
  }
  const double* dsrc = (side == 0 ? env->dL : env->dR) + so.blocks[b].off;
  if (cudaSetDevice(env->device) != cudaSuccess ||
      cudaMemcpy(out, dsrc, sizeof(double) * size_t(rows) * cols, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SU2_ECUDA;
  return SU2_OK;
}

int su2_env_destroy(su2_env* env) {
  if (!env) return SU2_EINVAL;
  env_free_device(env);
  delete env;
  return SU2_OK;
}

int su2_apply_heff(su2_ctx* ctx, const su2_env* env_c, const double* psi_in, double* psi_out, int32_t prec) {
  if (!ctx || !env_c || !psi_in || !psi_out) return fail(ctx, SU2_EINVAL, "null argument");
  su2_env* env = const_cast<su2_env*>(env_c);
  if (env->ctx != ctx) return fail(ctx, SU2_EINVAL, "environment belongs to another context");
  if ((uintptr_t(psi_in) | uintptr_t(psi_out)) & 7) return fail(ctx, SU2_EINVAL, "psi pointers must be 8-byte aligned");
  const int64_t n = env->psi_len;
  if (psi_in < psi_out + n && psi_out < psi_in + n) return fail(ctx, SU2_EINVAL, "psi_in and psi_out overlap");
  int rc = set_device(ctx);
  if (rc) return rc;
  if (prec == SU2_SPLIT_BF16) {
    std::string err;
    rc = split_apply(env, psi_in, psi_out, err);
    return rc ? fail(ctx, rc, err) : SU2_OK;
  }
  if (prec == SU2_SPLIT_FP8) return fail(ctx, SU2_EINVAL, "FP8 slices are not built (SU2_SPLIT_FP8 is reserved)");
  if (prec != SU2_FP64) return fail(ctx, SU2_EINVAL, "unknown precision");
  CUDA_TRY(ctx, cudaMemsetAsync(psi_out, 0, size_t(n) * sizeof(double), ctx->stream));
  if (env->os.on) stream_begin(env->os, ctx->stream);
  for (size_t ci = 0; ci < env->chunks.size(); ++ci) {
    if (env->os.on) stream_wait(env->os, int(ci), ctx->stream);
    launch_heff_fp64(ctx->stream, env->dL, env->dR, psi_in, psi_out, env->dT, env->dk1, env->dk2, env->dk2t,
                     env->chunks[ci], n, &env->prof);
    if (env->os.on) stream_release(env->os, int(ci), ctx->stream);
  }
  if (env->os.on) stream_end(env->os, ctx->stream);
  CUDA_TRY(ctx, cudaGetLastError());
  return SU2_OK;
}

int su2_apply_heff_host(su2_ctx* ctx, const su2_env* env_c, const double* in_h, double* out_h, int32_t prec) {
  if (!ctx || !env_c || !in_h || !out_h) return fail(ctx, SU2_EINVAL, "null argument");
  su2_env* env = const_cast<su2_env*>(env_c);
  int rc = set_device(ctx);
  if (rc) return rc;
  const size_t bytes = size_t(env->psi_len) * sizeof(double);
  if (!env->d_in_scratch) {
    rc = dev_alloc(ctx, &env->d_in_scratch, size_t(env->psi_len));
    if (!rc) rc = dev_alloc(ctx, &env->d_out_scratch, size_t(env->psi_len));
    if (rc) return rc;
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(env->d_in_scratch, in_h, bytes, cudaMemcpyHostToDevice, ctx->stream));
  rc = su2_apply_heff(ctx, env, env->d_in_scratch, env->d_out_scratch, prec);
  if (rc) return rc;
  CUDA_TRY(ctx, cudaMemcpyAsync(out_h, env->d_out_scratch, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return device_status_rc(ctx);
}

int su2_hash_group(int32_t id, int32_t step, int64_t group_count, int64_t i, int64_t* group) {
  if (!group || step < 1 || id < 0 || id >= step || group_count < 1 || i < 0) return SU2_EINVAL;
  int64_t a = group_count, b = step;
  while (b) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  const int64_t cycle_len = group_count / a;
  const int64_t cycle = i / cycle_len;
  // (id + step i + cycle) mod group_count without overflow for large i
  const int64_t si = int64_t((__int128)step * i % group_count);
  *group = ((int64_t(id) % group_count) + si + cycle % group_count) % group_count;
  return SU2_OK;
}

int su2_profile_enable(su2_env* env, int32_t on) {
  if (!env) return SU2_EINVAL;
  env->prof.drain();
  env->prof.on = on != 0;
  return SU2_OK;
}

int su2_profile_reset(su2_env* env) {
  if (!env) return SU2_EINVAL;
  env->prof.reset();
  return SU2_OK;
}

int su2_profile_read(su2_env* env, int32_t kind, int64_t* launches, double* ms, double* flops, const char** name) {
  static const char* names[kProfKinds] = {"k1_fp64", "k2_fp64", "split_slices", "k1_split", "k2_split",
                                          "kernel_launches"};
  if (!env || kind < 0 || kind >= kProfKinds) return SU2_EINVAL;
  env->prof.drain();
  if (launches) *launches = env->prof.launches[kind];
  if (ms) *ms = env->prof.ms[kind];
  if (flops) *flops = env->prof.flops[kind];
  if (name) *name = names[kind];
  return SU2_OK;
}

int su2_diag_heff(su2_ctx* ctx, const su2_env* env, double* diag_dev) {
  if (!ctx || !env || !diag_dev) return fail(ctx, SU2_EINVAL, "null argument");
  int rc = set_device(ctx);
  if (rc) return rc;
  const double* Ld = env->os.on ? env->os.ddiag : env->dL;
  const double* Rd = env->os.on ? env->os.ddiag : env->dR;
  launch_diag(ctx->stream, Ld, Rd, diag_dev, env->ddj, int64_t(env->dj.size()), env->ddt, env->psi_len);
  CUDA_TRY(ctx, cudaGetLastError());
  return SU2_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ Davidson
struct su2_dav {
  su2_ctx* ctx = nullptr;
  int device = -1;  // kept so that destroying the solver never reads its context
  const su2_env* env = nullptr;
  su2_dav_opts o{};
  int64_t n = 0;
  double *V = nullptr, *AV = nullptr, *x = nullptr, *ax = nullptr, *r = nullptr, *t = nullptr, *tmp = nullptr,
         *diag = nullptr;
  double *Hsub = nullptr, *Y = nullptr, *w = nullptr, *h = nullptr, *partial = nullptr, *scal = nullptr;
  int64_t* pidx = nullptr;
  double* host = nullptr;  // pinned: theta, nrm2
  int nsub = 0, iters = 0;
  double theta = 0.0, res = 0.0;
  bool converged = false;
  // graph mode: the subspace size lives on the device and one iteration
  // (H.v included) is a captured CUDA graph replayed on a private stream
  bool use_graph = false, graph_ready = false;
  int* d_nsub = nullptr;
  double *w_in = nullptr, *w_out = nullptr;
  cudaStream_t gstream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

static void dav_free(su2_dav* d) {
  if (d->device >= 0) cudaSetDevice(d->device);
  if (d->gexec) cudaGraphExecDestroy(d->gexec);
  if (d->graph) cudaGraphDestroy(d->graph);
  if (d->gstream) cudaStreamDestroy(d->gstream);
  if (d->ev_in) cudaEventDestroy(d->ev_in);
  if (d->ev_out) cudaEventDestroy(d->ev_out);
  cudaFree(d->d_nsub);
  cudaFree(d->w_in);
  cudaFree(d->w_out);
  double* ps[] = {d->V, d->AV, d->x, d->ax, d->r, d->t, d->tmp, d->diag, d->Hsub, d->Y, d->w, d->h, d->partial, d->scal};
  for (double* p : ps) cudaFree(p);
  cudaFree(d->pidx);
  if (d->host) cudaFreeHost(d->host);
}

extern "C" {

int su2_davidson_create(su2_ctx* ctx, const su2_env* env, const double* psi0, const su2_dav_opts* opts,
                        su2_dav** out) {
  if (!ctx || !env || !psi0 || !out) return fail(ctx, SU2_EINVAL, "null argument");
  *out = nullptr;
  int rc = set_device(ctx);
  if (rc) return rc;
  su2_dav* d = new (std::nothrow) su2_dav();
  if (!d) return fail(ctx, SU2_ENOMEM, "host allocation");
  d->ctx = ctx;
  d->device = ctx->device;
  d->env = env;
  d->o.tol = 1e-8;
  d->o.max_sub = 24;
  d->o.keep = 2;
  d->o.max_iter = 200;
  d->o.prec = SU2_FP64;
  if (opts) {
    if (opts->tol > 0) d->o.tol = opts->tol;
    if (opts->max_sub > 0) d->o.max_sub = opts->max_sub;
    if (opts->keep > 0) d->o.keep = opts->keep;
    if (opts->max_iter > 0) d->o.max_iter = opts->max_iter;
    d->o.prec = opts->prec;
    d->use_graph = opts->use_graph != 0;
  }
  if (d->o.prec != SU2_FP64 && d->o.prec != SU2_SPLIT_BF16) {
    const bool fp8 = d->o.prec == SU2_SPLIT_FP8;
    delete d;
    return fail(ctx, SU2_EINVAL, fp8 ? "FP8 slices are not built (SU2_SPLIT_FP8 is reserved)" : "unknown precision");
  }
  if (d->use_graph && env->os.on) {
    delete d;
    return fail(ctx, SU2_EINVAL, "graph capture of an environment with out-of-core operators is not supported");
  }
  if (d->o.max_sub > 32 || d->o.max_sub < 3 || d->o.keep >= d->o.max_sub) {
    delete d;
    return fail(ctx, SU2_EINVAL, "max_sub must be in [3, 32] and keep < max_sub");
  }
  const int64_t n = env->psi_len;
  d->n = n;
  const int ms = d->o.max_sub;
  const int ng = dav_grid(n);
  rc = dev_alloc(ctx, &d->V, size_t(ms) * n);
  if (!rc) rc = dev_alloc(ctx, &d->AV, size_t(ms) * n);
  if (!rc) rc = dev_alloc(ctx, &d->x, size_t(n));
  if (!rc) rc = dev_alloc(ctx, &d->ax, size_t(n));
  if (!rc) rc = dev_alloc(ctx, &d->r, size_t(n));
  if (!rc) rc = dev_alloc(ctx, &d->t, size_t(n));
  if (!rc) rc = dev_alloc(ctx, &d->tmp, size_t(2 * d->o.keep) * n);
  if (!rc) rc = dev_alloc(ctx, &d->diag, size_t(n));
  if (!rc) rc = dev_alloc(ctx, &d->Hsub, size_t(32 * 32));
  if (!rc) rc = dev_alloc(ctx, &d->Y, size_t(32 * 32));
  if (!rc) rc = dev_alloc(ctx, &d->w, size_t(32));
  if (!rc) rc = dev_alloc(ctx, &d->h, size_t(32));
  if (!rc) rc = dev_alloc(ctx, &d->partial, size_t(ng) * 32);
  if (!rc) rc = dev_alloc(ctx, &d->scal, size_t(8));
  if (!rc) rc = dev_alloc(ctx, &d->pidx, size_t(ng));
  if (!rc && cudaMallocHost(&d->host, 4 * sizeof(double)) != cudaSuccess) rc = fail(ctx, SU2_ENOMEM, "pinned host");
  if (!rc && d->use_graph) {
    rc = dev_alloc(ctx, &d->d_nsub, 1);
    if (!rc) rc = dev_alloc(ctx, &d->w_in, size_t(n));
    if (!rc) rc = dev_alloc(ctx, &d->w_out, size_t(n));
    if (!rc && (cudaStreamCreateWithFlags(&d->gstream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&d->ev_in, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&d->ev_out, cudaEventDisableTiming) != cudaSuccess))
      rc = fail(ctx, SU2_ECUDA, "graph stream/events");
  }
  if (rc) {
    dav_free(d);
    delete d;
    return rc;
  }
  cudaStream_t s = ctx->stream;
  rc = su2_diag_heff(ctx, env, d->diag);
  if (rc) {
    dav_free(d);
    delete d;
    return rc;
  }
  // V0 = psi0 / ||psi0||
  dav_multidot(s, psi0, n, 1, psi0, n, d->partial, d->scal, 1.0);
  dav_scale(s, d->V, psi0, d->scal, n);
  cudaMemsetAsync(d->Hsub, 0, 32 * 32 * sizeof(double), s);
  d->nsub = 1;
  if (d->use_graph) {
    const int one = 1;
    cudaMemcpyAsync(d->d_nsub, &one, sizeof(int), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  if (cudaGetLastError() != cudaSuccess) {
    dav_free(d);
    delete d;
    return fail(ctx, SU2_ECUDA, "davidson setup launch");
  }
  *out = d;
  return SU2_OK;
}

// one Davidson iteration with the subspace size on the device, recorded on
// stream s (for capture); results land in the pinned host buffer
static int dav_record_iteration(su2_ctx* ctx, su2_dav* d, cudaStream_t s) {
  const int64_t n = d->n;
  const int ld = 32;
  dav_newest(s, d->V, n, d->d_nsub, d->w_in, 0);
  int rc = su2_apply_heff(ctx, d->env, d->w_in, d->w_out, d->o.prec);
  if (rc) return rc;
  dav_newest(s, d->AV, n, d->d_nsub, d->w_out, 1);
  dav_multidot(s, d->V, n, 0, d->w_out, n, d->partial, d->h, 1.0, d->d_nsub);
  dav_copy_col(s, d->Hsub, ld, 0, d->h, 0, d->d_nsub);
  dav_jacobi(s, d->Hsub, ld, 0, d->w, d->Y, ctx->d_status, d->d_nsub);
  dav_combine(s, d->V, d->AV, n, 0, d->Y, n, d->x, d->ax, d->d_nsub);
  dav_residual(s, d->x, d->ax, d->w, n, d->r);
  dav_multidot(s, d->r, n, 1, d->r, n, d->partial, d->scal, 1.0);
  dav_precond(s, d->r, d->diag, d->w, n, d->t);
  dav_restart(s, d->V, d->AV, n, d->Y, ld, d->Hsub, d->w, d->o.keep, d->o.max_sub, d->d_nsub, d->tmp);
  for (int pass = 0; pass < 2; ++pass) {
    dav_multidot(s, d->V, n, 0, d->t, n, d->partial, d->h, 1.0, d->d_nsub);
    dav_subtract(s, d->V, n, 0, d->h, n, d->t, d->d_nsub);
  }
  dav_multidot(s, d->t, n, 1, d->t, n, d->partial, d->scal + 1, 1.0);
  dav_append(s, d->V, n, d->d_nsub, d->t, d->scal + 1);
  cudaMemcpyAsync(d->host, d->w, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(d->host + 1, d->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  return SU2_OK;
}

static int dav_graph_step(su2_ctx* ctx, su2_dav* d) {
  if (!d->graph_ready) {
    su2_env* env = const_cast<su2_env*>(d->env);
    const bool prof_on = env->prof.on;
    env->prof.drain();
    env->prof.on = false;
    cudaStream_t saved = ctx->stream;
    ctx->stream = d->gstream;
    CUDA_TRY(ctx, cudaStreamBeginCapture(d->gstream, cudaStreamCaptureModeThreadLocal));
    int rc = dav_record_iteration(ctx, d, d->gstream);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(d->gstream, &g);
    ctx->stream = saved;
    env->prof.on = prof_on;
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ce != cudaSuccess) return fail(ctx, SU2_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    d->graph = g;
    CUDA_TRY(ctx, cudaGraphInstantiate(&d->gexec, d->graph, 0));
    d->graph_ready = true;
  }
  CUDA_TRY(ctx, cudaEventRecord(d->ev_in, ctx->stream));
  CUDA_TRY(ctx, cudaStreamWaitEvent(d->gstream, d->ev_in, 0));
  CUDA_TRY(ctx, cudaGraphLaunch(d->gexec, d->gstream));
  CUDA_TRY(ctx, cudaEventRecord(d->ev_out, d->gstream));
  CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, d->ev_out, 0));
  CUDA_TRY(ctx, cudaStreamSynchronize(d->gstream));
  return SU2_OK;
}

int su2_davidson_step(su2_ctx* ctx, su2_dav* d, double* theta, double* resnorm) {
  if (!ctx || !d || d->ctx != ctx) return fail(ctx, SU2_EINVAL, "null argument");
  int rc = set_device(ctx);
  if (rc) return rc;
  if (d->use_graph) {
    if (d->converged) {
      if (theta) *theta = d->theta;
      if (resnorm) *resnorm = d->res;
      return SU2_OK;
    }
    rc = dav_graph_step(ctx, d);
    if (rc) return rc;
    rc = device_status_rc(ctx);
    if (rc) return rc;
    d->iters += 1;
    d->theta = d->host[0];
    d->res = std::sqrt(std::max(0.0, d->host[1]));
    if (theta) *theta = d->theta;
    if (resnorm) *resnorm = d->res;
    if (d->res <= d->o.tol || !(d->host[2] > 1e-28)) d->converged = true;
    return SU2_OK;
  }
  cudaStream_t s = ctx->stream;
  const int64_t n = d->n;
  const int ms = d->o.max_sub, ld = 32;
  if (d->converged) {
    if (theta) *theta = d->theta;
    if (resnorm) *resnorm = d->res;
    return SU2_OK;
  }
  const int j = d->nsub - 1;  // newest vector
  rc = su2_apply_heff(ctx, d->env, d->V + int64_t(j) * n, d->AV + int64_t(j) * n, d->o.prec);
  if (rc) return rc;
  dav_multidot(s, d->V, n, d->nsub, d->AV + int64_t(j) * n, n, d->partial, d->h, 1.0);
  dav_copy_col(s, d->Hsub, ld, j, d->h, d->nsub);
  dav_jacobi(s, d->Hsub, ld, d->nsub, d->w, d->Y, ctx->d_status);
  dav_combine(s, d->V, d->AV, n, d->nsub, d->Y, n, d->x, d->ax);
  dav_residual(s, d->x, d->ax, d->w, n, d->r);
  dav_multidot(s, d->r, n, 1, d->r, n, d->partial, d->scal, 1.0);
  CUDA_TRY(ctx, cudaMemcpyAsync(d->host, d->w, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(ctx, cudaMemcpyAsync(d->host + 1, d->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(ctx, cudaStreamSynchronize(s));
  rc = device_status_rc(ctx);
  if (rc) return rc;
  d->iters += 1;
  d->theta = d->host[0];
  d->res = std::sqrt(std::max(0.0, d->host[1]));
  if (theta) *theta = d->theta;
  if (resnorm) *resnorm = d->res;
  if (d->res <= d->o.tol) {
    d->converged = true;
    return SU2_OK;
  }
  dav_precond(s, d->r, d->diag, d->w, n, d->t);
  if (d->nsub >= ms) {  // restart on the lowest Ritz vectors
    const int keep = d->o.keep;
    for (int q = 0; q < keep; ++q)
      dav_combine(s, d->V, d->AV, n, d->nsub, d->Y + q * ld, n, d->tmp + int64_t(2 * q) * n,
                  d->tmp + int64_t(2 * q + 1) * n);
    for (int q = 0; q < keep; ++q) {
      cudaMemcpyAsync(d->V + int64_t(q) * n, d->tmp + int64_t(2 * q) * n, n * sizeof(double),
                      cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d->AV + int64_t(q) * n, d->tmp + int64_t(2 * q + 1) * n, n * sizeof(double),
                      cudaMemcpyDeviceToDevice, s);
    }
    dav_diag_set(s, d->Hsub, ld, keep, d->w);
    d->nsub = keep;
  }
  for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
    dav_multidot(s, d->V, n, d->nsub, d->t, n, d->partial, d->h, 1.0);
    dav_subtract(s, d->V, n, d->nsub, d->h, n, d->t);
  }
  dav_multidot(s, d->t, n, 1, d->t, n, d->partial, d->scal, 1.0);
  CUDA_TRY(ctx, cudaMemcpyAsync(d->host + 2, d->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (!(d->host[2] > 1e-28)) {  // correction vanished: nothing left to add
    d->converged = true;
    return SU2_OK;
  }
  dav_scale(s, d->V + int64_t(d->nsub) * n, d->t, d->scal, n);
  d->nsub += 1;
  CUDA_TRY(ctx, cudaGetLastError());
  return SU2_OK;
}

int su2_davidson_solve(su2_ctx* ctx, su2_dav* d, double* theta, double* resnorm, int32_t* iterations) {
  if (!ctx || !d) return fail(ctx, SU2_EINVAL, "null argument");
  while (!d->converged && d->iters < d->o.max_iter) {
    int rc = su2_davidson_step(ctx, d, theta, resnorm);
    if (rc) return rc;
  }
  if (theta) *theta = d->theta;
  if (resnorm) *resnorm = d->res;
  if (iterations) *iterations = d->iters;
  return d->converged ? SU2_OK : fail(ctx, SU2_ENOTCONV, "Davidson iteration limit reached");
}

int su2_energy(const su2_dav* d, double* E) {
  if (!d || !E) return SU2_EINVAL;
  *E = d->theta;
  return SU2_OK;
}

int su2_energy_check(su2_ctx* ctx, su2_dav* d, int32_t prec, double* rq, double* resnorm) {
  if (!ctx || !d || d->ctx != ctx || !rq) return fail(ctx, SU2_EINVAL, "null argument");
  if (prec != SU2_FP64 && prec != SU2_SPLIT_BF16) return fail(ctx, SU2_EINVAL, "unknown precision");
  int rc = set_device(ctx);
  if (rc) return rc;
  cudaStream_t s = ctx->stream;
  const int64_t n = d->n;
  double* hx = nullptr;
  double* r = nullptr;
  rc = dev_alloc(ctx, &hx, size_t(n));
  if (!rc) rc = dev_alloc(ctx, &r, size_t(n));
  if (!rc) rc = su2_apply_heff(ctx, d->env, d->x, hx, prec);
  double xs[2] = {0.0, 0.0}, rr = 0.0;
  if (!rc) {
    dav_multidot(s, d->x, n, 1, d->x, n, d->partial, d->scal, 1.0);   // <x|x>
    dav_multidot(s, d->x, n, 1, hx, n, d->partial, d->scal + 1, 1.0);  // <x|Hx>
    if (cudaMemcpyAsync(xs, d->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = fail(ctx, SU2_ECUDA, "energy check: reading the dot products");
  }
  if (!rc) rc = device_status_rc(ctx);
  if (!rc && !(xs[0] > 0.0)) rc = fail(ctx, SU2_EINVAL, "energy check: the Ritz vector is zero");
  if (!rc) {
    *rq = xs[1] / xs[0];
    if (resnorm) {
      // ||Hx - rq x|| / ||x||
      if (cudaMemcpyAsync(d->scal + 2, rq, sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = fail(ctx, SU2_ECUDA, "energy check: upload");
      if (!rc) {
        dav_residual(s, d->x, hx, d->scal + 2, n, r);
        dav_multidot(s, r, n, 1, r, n, d->partial, d->scal + 3, 1.0);
        if (cudaMemcpyAsync(&rr, d->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
          rc = fail(ctx, SU2_ECUDA, "energy check: reading the residual");
      }
      if (!rc) *resnorm = std::sqrt(std::max(0.0, rr) / xs[0]);
    }
  }
  cudaStreamSynchronize(s);
  cudaFree(hx);
  cudaFree(r);
  return rc;
}

int su2_davidson_vector(su2_ctx* ctx, su2_dav* d, double* x_dev) {
  if (!ctx || !d || !x_dev) return fail(ctx, SU2_EINVAL, "null argument");
  int rc = set_device(ctx);
  if (rc) return rc;
  cudaStream_t s = ctx->stream;
  const int64_t n = d->n;
  int ng = 0;
  dav_absmax(s, d->x, n, d->partial, d->pidx, &ng);
  std::vector<double> pv(ng);
  std::vector<int64_t> pi(ng);
  CUDA_TRY(ctx, cudaMemcpyAsync(pv.data(), d->partial, ng * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(ctx, cudaMemcpyAsync(pi.data(), d->pidx, ng * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(ctx, cudaStreamSynchronize(s));
  int best = 0;
  for (int g = 1; g < ng; ++g)
    if (pv[g] > pv[best] || (pv[g] == pv[best] && pi[g] < pi[best])) best = g;
  double xv = 0.0;
  CUDA_TRY(ctx, cudaMemcpy(&xv, d->x + pi[best], sizeof(double), cudaMemcpyDeviceToHost));
  // x has unit norm up to rounding; scale by +-1 / ||x||
  dav_multidot(s, d->x, n, 1, d->x, n, d->partial, d->scal, 1.0);
  double nrm2 = 0.0;
  CUDA_TRY(ctx, cudaMemcpyAsync(&nrm2, d->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(ctx, cudaStreamSynchronize(s));
  const double sgn_nrm2 = nrm2;  // positive
  dav_scale(s, x_dev, d->x, d->scal, n);
  if (xv < 0) {
    double m1 = -1.0;
    double* dm = d->h;
    CUDA_TRY(ctx, cudaMemcpyAsync(dm, &m1, sizeof(double), cudaMemcpyHostToDevice, s));
    dav_combine(s, x_dev, nullptr, n, 1, dm, n, x_dev, nullptr);
  }
  (void)sgn_nrm2;
  CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return SU2_OK;
}

int su2_davidson_destroy(su2_dav* d) {
  if (!d) return SU2_EINVAL;
  dav_free(d);
  delete d;
  return SU2_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ two-site sweep
struct su2_sweep {
  su2_ctx* ctx = nullptr;
  int device = -1;
  su2::SweepBlocks* w = nullptr;
  int L = 0, N = 0;
  su2_sweep_opts o{};
  int pos = 0, dir = 1;  // next window and direction
  int64_t steps = 0;
  std::vector<double> guess;  // predicted start vector of the next window (empty: seeded)
  // Heisenberg chain (spin-1/2 sites): blocks and the MPS tensors that grew
  // them, on the host (hL[i]: the first i sites, hR[k]: the last k sites)
  bool heis = false;
  su2_hamiltonian H{};
  std::vector<HeisBlock> hL, hR;
  std::vector<std::vector<std::vector<double>>> hLq, hRq;
};

extern "C" {

int su2_sweep_create(su2_ctx* ctx, const su2_hamiltonian* H, const su2_bond_chain* right_chain, int32_t N,
                     const su2_sweep_opts* opts, su2_sweep** out) {
  if (!ctx || !H || !right_chain || !opts || !out) return fail(ctx, SU2_EINVAL, "null argument");
  *out = nullptr;
  if (ctx->device < 0) return fail(ctx, SU2_EINVAL, "the sweep needs a device context");
  const bool heis = H->model == SU2_MODEL_HEISENBERG;
  if (!heis && (H->model != SU2_MODEL_AB_INITIO || !H->h || !H->eri))
    return fail(ctx, SU2_EINVAL, "the sweep needs the ab initio model (with its integrals) or the Heisenberg chain");
  if (opts->D < 1 || N < 0) return fail(ctx, SU2_EINVAL, "D must be >= 1");
  if (opts->twoS < 0) return fail(ctx, SU2_EINVAL, "the target spin must be >= 0");
  if (opts->prec != SU2_FP64 && opts->prec != SU2_SPLIT_BF16) return fail(ctx, SU2_EINVAL, "unknown precision");
  std::vector<std::vector<Sector>> rch;
  if (right_chain->n_bonds < 1 || !right_chain->bond_offset || !right_chain->sectors)
    return fail(ctx, SU2_EINVAL, "bad bond chain");
  for (int k = 0; k < right_chain->n_bonds; ++k) {
    std::vector<Sector> v;
    for (int i = right_chain->bond_offset[k]; i < right_chain->bond_offset[k + 1]; ++i)
      v.push_back(Sector{right_chain->sectors[i].N, right_chain->sectors[i].twoS, right_chain->sectors[i].dim});
    rch.push_back(v);
  }
  int rc = set_device(ctx);
  if (rc) return rc;
  su2_sweep* sw = new (std::nothrow) su2_sweep();
  if (!sw) return fail(ctx, SU2_ENOMEM, "host allocation");
  sw->ctx = ctx;
  sw->device = ctx->device;
  sw->L = H->n_left + 2 + H->n_right;
  sw->N = N;
  sw->o = *opts;
  if (sw->o.tol <= 0) sw->o.tol = 1e-8;
  if (sw->o.max_iter <= 0) sw->o.max_iter = 400;
  if (sw->o.n_slices <= 0) sw->o.n_slices = 5;
  std::string err;
  if (heis) {
    // initial right blocks grown site by site by the caller's tensors or the seeded ones
    const int L = sw->L;
    sw->heis = true;
    sw->H = *H;
    sw->H.h = sw->H.eri = sw->H.mps_left = sw->H.mps_right = nullptr;
    if (int(rch.size()) != L - 1) err = "the initial right chain must hold the bonds of 0 .. L-2 sites";
    sw->hL.resize(size_t(L - 1));
    sw->hR.resize(size_t(L - 1));
    sw->hLq.resize(size_t(L - 1));
    sw->hRq.resize(size_t(L - 1));
    if (err.empty()) sw->hR[0].sec = rch[0];
    std::vector<int> sN, sS;
    site_states(SU2_SITE_SPIN_HALF, sN, sS);
    size_t pos = 0;
    for (int k = 1; k < L - 1 && err.empty(); ++k) {
      const auto& prev = rch[size_t(k - 1)];
      const auto& cur = rch[size_t(k)];
      std::vector<std::vector<double>> Q(cur.size());
      for (size_t qo = 0; qo < cur.size() && err.empty(); ++qo) {
        int r0 = 0;
        for (const Sector& p : prev)
          for (size_t si = 0; si < sN.size(); ++si)
            if (p.N + sN[si] == cur[qo].N && triangle(p.twoS, sS[si], cur[qo].twoS)) r0 += p.dim;
        if (r0 < cur[qo].dim) {
          err = "bond dimension exceeds the states available from the previous bond";
        } else if (H->mps_right) {
          const size_t n = size_t(r0) * size_t(cur[qo].dim);
          Q[qo].assign(H->mps_right + pos, H->mps_right + pos + n);
          pos += n;
        } else {
          Q[qo] = seeded_mps_tensor(H->seed, 3, k, int(qo), r0, cur[qo].dim);
        }
      }
      if (err.empty()) err = heis_grow(sw->hR[size_t(k - 1)], cur, Q, false, H->J, sw->hR[size_t(k)]);
      sw->hRq[size_t(k)] = std::move(Q);
    }
  } else {
    sw->w = sweep_init(*H, rch, ctx->device, ctx->stream, 0, err);
  }
  if (!err.empty()) {
    delete sw;
    return fail(ctx, SU2_EINVAL, err);
  }
  *out = sw;
  return SU2_OK;
}

int su2_sweep_run(su2_ctx* ctx, su2_sweep* sw, int32_t n_steps, double* energies, double* discarded,
                  int32_t* iterations, double* start_energies) {
  if (!ctx || !sw || sw->ctx != ctx || n_steps < 0) return fail(ctx, SU2_EINVAL, "null argument");
  int rc = set_device(ctx);
  if (rc) return rc;
  const int L = sw->L;
  for (int k = 0; k < n_steps; ++k) {
    const int i = sw->pos;
    const int kind = sw->heis ? SU2_SITE_SPIN_HALF : SU2_SITE_ORBITAL;
    su2_sectors S;
    S.site_kind = kind;
    S.N = sw->N;
    S.twoS = sw->o.twoS;
    su2_env* env = new (std::nothrow) su2_env();
    if (!env) return fail(ctx, SU2_ENOMEM, "host allocation");
    env->ctx = ctx;
    env->device = ctx->device;
    std::string err;
    if (sw->heis) {
      const HeisBlock& lb = sw->hL[size_t(i)];
      const HeisBlock& rb = sw->hR[size_t(L - 2 - i)];
      env->table = make_table(sw->H, kind);
      err = heis_side_ops(env->table, true, lb, env->L);
      if (err.empty()) err = heis_side_ops(env->table, false, rb, env->R);
      S.left = lb.sec;
      S.right = rb.sec;
    } else {
      err = sweep_env(sw->w, i, env->table, env->L, env->R, S.left, S.right);
    }
    if (err.empty()) build_blocks(S.left, S.right, kind, sw->N, S.twoS, S.blocks, S.psi_len);
    if (err.empty() && S.psi_len == 0) err = "no two-site state with the target particle number";
    if (err.empty()) {
      env->psi_len = S.psi_len;
      env->blocks = S.blocks;
      env->lsec = S.left;
      env->rsec = S.right;
      err = build_tasks(env->table, S.left, S.right, S.blocks, S.twoS, env->L, env->R, env->tasks);
    }
    if (!err.empty()) {
      cudaFree(env->L.dev_ready);
      cudaFree(env->R.dev_ready);
      delete env;
      return fail(ctx, SU2_EINVAL, err);
    }
    su2_env_opts eo{};
    eo.prepare_split = sw->o.prec == SU2_SPLIT_BF16;
    eo.n_slices = sw->o.n_slices;
    rc = finish_env(ctx, env, &S, &eo);
    if (rc) return rc;
    // Davidson from the predicted start vector, else from a seeded one
    const int64_t n = S.psi_len;
    std::vector<double> h(static_cast<size_t>(n));
    double gn = 0.0;
    if (sw->o.predict && int64_t(sw->guess.size()) == n)
      for (double v : sw->guess) gn += v * v;
    if (gn > 0.0) {
      h.swap(sw->guess);
    } else {
      const uint64_t key = block_key(sw->o.guess_seed, 9, uint64_t(sw->steps), 0, 0);
      for (int64_t x = 0; x < n; ++x) h[size_t(x)] = uniform_elem(key, uint64_t(x));
    }
    sw->guess.clear();
    double* d0 = nullptr;
    double* dx = nullptr;
    rc = dev_alloc(ctx, &d0, size_t(n));
    if (!rc) rc = dev_alloc(ctx, &dx, size_t(n));
    if (!rc && cudaMemcpy(d0, h.data(), size_t(n) * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = fail(ctx, SU2_ECUDA, "upload");
    su2_dav* dav = nullptr;
    double theta = 0.0, res = 0.0, theta0 = 0.0;
    int32_t its = 0;
    if (!rc) {
      su2_dav_opts dop{sw->o.tol, 24, 2, sw->o.max_iter, sw->o.prec, 0};
      rc = su2_davidson_create(ctx, env, d0, &dop, &dav);
    }
    // the first iteration's Ritz value is the Rayleigh quotient of the start vector
    if (!rc) rc = su2_davidson_step(ctx, dav, &theta0, &res);
    if (!rc) {
      rc = su2_davidson_solve(ctx, dav, &theta, &res, &its);
      if (rc == SU2_ENOTCONV) rc = SU2_OK;  // the energy of the last iterate is reported
    }
    if (!rc) rc = su2_davidson_vector(ctx, dav, dx);
    if (!rc && cudaMemcpy(h.data(), dx, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = fail(ctx, SU2_ECUDA, "download");
    if (dav) su2_davidson_destroy(dav);
    cudaFree(d0);
    cudaFree(dx);
    env_free_device(env);
    delete env;
    if (rc) return rc;
    if (energies) energies[k] = theta;
    if (iterations) iterations[k] = its;
    if (start_energies) start_energies[k] = theta0;
    // truncate and grow the block on the side the sweep moves to; predict
    // the next window's start vector (at a turn the next window is this one)
    double w = 0.0;
    const bool grow = sw->dir > 0 ? i < L - 2 : i > 0;
    if (grow) {
      std::vector<Sector> cur;
      std::vector<std::vector<double>> Q, rest;
      err = sweep_split(S.blocks, h.data(), S.left, S.right, sw->N, sw->o.D, sw->dir > 0, cur, Q, &w,
                        sw->o.predict ? &rest : nullptr, kind, S.twoS);
      if (err.empty() && sw->heis) {
        // the grown block on the host, then the next window's guess
        if (sw->dir > 0) {
          err = heis_grow(sw->hL[size_t(i)], cur, Q, true, sw->H.J, sw->hL[size_t(i + 1)]);
          sw->hLq[size_t(i + 1)] = Q;
          if (err.empty() && sw->o.predict)
            err = predict_guess(true, S.left, S.right, sw->hL[size_t(i + 1)].sec, sw->hR[size_t(L - 3 - i)].sec,
                                sw->hRq[size_t(L - 2 - i)], sw->N, kind, cur, rest, sw->guess, S.twoS);
        } else {
          err = heis_grow(sw->hR[size_t(L - 2 - i)], cur, Q, false, sw->H.J, sw->hR[size_t(L - 1 - i)]);
          sw->hRq[size_t(L - 1 - i)] = Q;
          if (err.empty() && sw->o.predict)
            err = predict_guess(false, S.left, S.right, sw->hL[size_t(i - 1)].sec, sw->hR[size_t(L - 1 - i)].sec,
                                sw->hLq[size_t(i)], sw->N, kind, cur, rest, sw->guess, S.twoS);
        }
      } else if (err.empty()) {
        err = sweep_grow(sw->w, i, sw->dir > 0, cur, Q);
        if (err.empty() && sw->o.predict)
          err = sweep_predict(sw->w, i, sw->dir > 0, S.left, S.right, sw->N, cur, rest, sw->guess, S.twoS);
      }
      if (!err.empty()) return fail(ctx, SU2_EINVAL, err);
    } else if (sw->o.predict) {
      sw->guess = h;
    }
    if (discarded) discarded[k] = w;
    sw->steps += 1;
    // next window: turn at the ends
    if (sw->dir > 0) {
      if (i == L - 2) sw->dir = -1;
      else sw->pos = i + 1;
    } else {
      if (i == 0) sw->dir = 1;
      else sw->pos = i - 1;
    }
  }
  return SU2_OK;
}

int su2_sweep_checkpoint(su2_ctx* ctx, su2_sweep* sw, int32_t* n_bonds, int32_t* n_sectors, int64_t* n_values,
                         int32_t* bond_offset, su2_sector* sectors, double* mps) {
  if (!ctx || !sw || sw->ctx != ctx || !n_bonds || !n_sectors || !n_values)
    return fail(ctx, SU2_EINVAL, "null argument");
  if (sw->pos != 0 || sw->dir != 1)
    return fail(ctx, SU2_EINVAL, "a checkpoint is taken at the start of a right-moving half-sweep (window 0)");
  std::vector<std::vector<Sector>> chain;
  std::vector<std::vector<std::vector<double>>> tensors;
  if (sw->heis) {
    for (size_t k = 0; k < sw->hR.size(); ++k) {
      chain.push_back(sw->hR[k].sec);
      tensors.push_back(k > 0 ? sw->hRq[k] : std::vector<std::vector<double>>());
    }
  } else {
    const std::string err = sweep_right_state(sw->w, chain, tensors);
    if (!err.empty()) return fail(ctx, SU2_EINVAL, err);
  }
  int32_t ns = 0;
  int64_t nv = 0;
  for (size_t k = 0; k < chain.size(); ++k) {
    ns += int32_t(chain[k].size());
    for (const auto& q : tensors[k]) nv += int64_t(q.size());
  }
  const bool sizes_only = !bond_offset && !sectors && !mps;
  if (!sizes_only && (!bond_offset || !sectors || !mps)) return fail(ctx, SU2_EINVAL, "null output array");
  if (!sizes_only && (*n_bonds < int32_t(chain.size()) || *n_sectors < ns || *n_values < nv))
    return fail(ctx, SU2_EINVAL, "output arrays smaller than the checkpoint");
  *n_bonds = int32_t(chain.size());
  *n_sectors = ns;
  *n_values = nv;
  if (sizes_only) return SU2_OK;
  int32_t at = 0;
  int64_t pos = 0;
  for (size_t k = 0; k < chain.size(); ++k) {
    bond_offset[k] = at;
    for (const Sector& q : chain[k]) sectors[at++] = su2_sector{q.N, q.twoS, q.dim};
    for (const auto& q : tensors[k]) {
      std::copy(q.begin(), q.end(), mps + pos);
      pos += int64_t(q.size());
    }
  }
  bond_offset[chain.size()] = at;
  return SU2_OK;
}

int su2_sweep_destroy(su2_sweep* sw) {
  if (!sw) return SU2_EINVAL;
  if (sw->device >= 0) cudaSetDevice(sw->device);
  if (sw->w) sweep_free(sw->w);
  delete sw;
  return SU2_OK;
}

}  // extern "C"
