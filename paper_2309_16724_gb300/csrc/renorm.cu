// Execution of renormalisation steps (su2_renorm.h): on the GPU the products
// F += v A E D^T run through the grouped FP64 kernels of the H.psi path
// (K1: T = E D^T once per distinct (E, D) pair, K2: output-stationary
// F += sum v A T, no atomics), the sums of operator blocks through a small
// kernel that walks each destination range once; on the host the same work
// runs as plain loops (host-only contexts).
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <unordered_map>

#include "su2_device.h"
#include "su2_renorm.h"

namespace su2 {
namespace {

constexpr int64_t kGroupChunk = 1 << 16;

struct GroupPiece {  // a piece of one destination range for one CTA
  int64_t dst, n0, n1;
  int32_t t0, t1;
};

__global__ void group_kernel(const GroupPiece* __restrict__ pieces, const RTerm* __restrict__ terms,
                             const double* __restrict__ src, double* __restrict__ dst) {
  const GroupPiece p = pieces[blockIdx.x];
  for (int64_t i = p.n0 + threadIdx.x; i < p.n1; i += blockDim.x) {
    double s = dst[p.dst + i];
    for (int t = p.t0; t < p.t1; ++t) s += terms[t].w * src[terms[t].src + i];
    dst[p.dst + i] = s;
  }
}

__global__ void ident_kernel(const RIdent* __restrict__ id, double* __restrict__ a) {
  const RIdent r = id[blockIdx.x];
  for (int i = threadIdx.x; i < r.d; i += blockDim.x) a[r.off + int64_t(i) * (r.d + 1)] = r.c;
}

std::vector<GroupPiece> pieces_of(const std::vector<RGroup>& g) {
  std::vector<GroupPiece> p;
  for (const RGroup& x : g)
    for (int64_t i = 0; i < x.n; i += kGroupChunk) p.push_back(GroupPiece{x.dst, i, std::min(x.n, i + kGroupChunk), x.t0, x.t1});
  return p;
}

template <class T>
cudaError_t upload(T** d, const std::vector<T>& h) {
  *d = nullptr;
  if (h.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(T));
  if (e == cudaSuccess) e = cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

class DeviceBackend : public RenormBackend {
 public:
  DeviceBackend(int device, void* stream, int64_t budget)
      : device_(device), s_((cudaStream_t)stream), budget_(budget > 0 ? budget : (int64_t(2) << 30)) {}
  ~DeviceBackend() override {
    cudaSetDevice(device_);
    cudaFree(cur_);
  }
  int64_t size() const override { return size_; }
  double* take_device() override {
    double* p = cur_;
    cur_ = nullptr;
    size_ = 0;
    return p;
  }

  std::string run(const RStep& st) override {
    double* out = nullptr;
    std::string err = run_keep(st, cur_, &out);
    if (!err.empty()) return err;
    cudaFree(cur_);
    cur_ = out;
    size_ = st.dst_size;
    return "";
  }

  std::string run_keep(const RStep& st, const double* old, double** out) override {
    *out = nullptr;
    std::string err;
    double *src = nullptr, *dst = nullptr, *q = nullptr, *T = nullptr;
    RIdent* did = nullptr;
    GroupPiece *dtp = nullptr, *dcp = nullptr;
    RTerm *dtt = nullptr, *dct = nullptr;
    K1Job* dk1 = nullptr;
    K2Job* dk2 = nullptr;
    K2Task* dk2t = nullptr;
    auto ck = [&](cudaError_t e, const char* what) {
      if (e != cudaSuccess && err.empty()) err = std::string("renormalisation: ") + what + ": " + cudaGetErrorString(e);
      return err.empty();
    };
    cudaSetDevice(device_);
    (void)cudaGetLastError();
    const int64_t srcn = std::max<int64_t>(st.src_size, 1), dstn = std::max<int64_t>(st.dst_size, 1);
    if (ck(cudaMalloc(&src, size_t(srcn) * sizeof(double)), "source arena") && st.old_size > 0)
      ck(cudaMemcpyAsync(src, old, size_t(st.old_size) * sizeof(double), cudaMemcpyDeviceToDevice, s_), "copy");
    if (err.empty() && st.src_size > st.old_size)
      ck(cudaMemsetAsync(src + st.old_size, 0, size_t(st.src_size - st.old_size) * sizeof(double), s_), "memset");
    if (err.empty() && !st.idents.empty() && ck(upload(&did, st.idents), "identities"))
      ident_kernel<<<unsigned(st.idents.size()), 128, 0, s_>>>(did, src);
    const auto tp = pieces_of(st.temps);
    if (err.empty() && !tp.empty() && ck(upload(&dtp, tp), "temps") && ck(upload(&dtt, st.temp_terms), "temp terms"))
      group_kernel<<<unsigned(tp.size()), 256, 0, s_>>>(dtp, dtt, src, src);
    if (err.empty()) ck(cudaStreamSynchronize(s_), "temporaries");
    if (err.empty()) ck(upload(&q, st.q), "Q arena");
    if (err.empty() && ck(cudaMalloc(&dst, size_t(dstn) * sizeof(double)), "destination arena"))
      ck(cudaMemsetAsync(dst, 0, size_t(dstn) * sizeof(double), s_), "memset");
    // the products, in chunks whose intermediates T fit the budget
    if (err.empty() && !st.tasks.empty()) {
      std::vector<int64_t> ord(st.tasks.size());
      for (size_t i = 0; i < ord.size(); ++i) ord[i] = int64_t(i);
      std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return st.tasks[a].f < st.tasks[b].f; });
      std::vector<K1Job> k1;
      std::vector<K2Job> k2;
      std::vector<K2Task> k2t;
      std::vector<Chunk> chunks;
      int64_t max_t = 0;
      size_t i = 0;
      while (i < ord.size()) {
        Chunk c{int64_t(k1.size()), 0, int64_t(k2.size()), 0, 0.0, 0.0};
        std::map<std::tuple<int64_t, int64_t, int32_t, int32_t, int32_t>, int64_t> toff;
        int64_t tsz = 0;
        size_t j = i;
        std::vector<K2Job> jobs;
        std::vector<double> cost;
        while (j < ord.size()) {
          const int64_t f = st.tasks[ord[j]].f;
          size_t e = j;
          int64_t add = 0;
          for (; e < ord.size() && st.tasks[ord[e]].f == f; ++e) {
            const RTask& t = st.tasks[ord[e]];
            if (!toff.count({t.e, t.d, t.k1, t.k2, t.n})) add += (int64_t(t.k1) * t.n + 1) & ~int64_t(1);
          }
          if (j > i && (tsz + add) * int64_t(sizeof(double)) > budget_) break;
          const int32_t tb = int32_t(k2t.size());
          double c2 = 0.0;
          for (size_t x = j; x < e; ++x) {
            const RTask& t = st.tasks[ord[x]];
            auto key = std::make_tuple(t.e, t.d, t.k1, t.k2, t.n);
            auto it = toff.find(key);
            if (it == toff.end()) {
              it = toff.emplace(key, tsz).first;
              for (int tc = 0; tc < (t.n + kTile - 1) / kTile; ++tc)
                for (int tr = 0; tr < (t.k1 + kTile - 1) / kTile; ++tr)
                  k1.push_back(K1Job{t.e, t.d, tsz, t.k1, t.k2, t.n, tr, tc, 0});
              tsz += (int64_t(t.k1) * t.n + 1) & ~int64_t(1);
              c.k1_flops += 2.0 * t.k1 * t.k2 * t.n;
            }
            K2Task kt;
            kt.a_off = t.a;
            kt.b_off = it->second;
            kt.k1 = t.k1;
            kt.flags = 0;
            kt.v = t.v;
            k2t.push_back(kt);
            c.k2_flops += 2.0 * t.m * t.k1 * t.n;
            c2 += t.k1;
          }
          const RTask& t0 = st.tasks[ord[j]];
          for (int tc = 0; tc < (t0.n + kTile - 1) / kTile; ++tc)
            for (int tr = 0; tr < (t0.m + kTile - 1) / kTile; ++tr) {
              jobs.push_back(K2Job{f, t0.m, t0.n, tr, tc, tb, int32_t(k2t.size())});
              cost.push_back(c2);
            }
          j = e;
        }
        std::vector<size_t> jo(jobs.size());
        for (size_t x = 0; x < jo.size(); ++x) jo[x] = x;
        std::stable_sort(jo.begin(), jo.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
        for (size_t x : jo) k2.push_back(jobs[x]);
        c.k1_end = int64_t(k1.size());
        c.k2_end = int64_t(k2.size());
        chunks.push_back(c);
        max_t = std::max(max_t, tsz);
        flops += c.k1_flops + c.k2_flops;
        i = j;
      }
      if (k2t.size() >= (size_t(1) << 31)) err = "renormalisation: too many products in one step";
      if (err.empty()) ck(cudaMalloc(&T, size_t(std::max<int64_t>(max_t, 2)) * sizeof(double)), "T");
      if (err.empty()) ck(upload(&dk1, k1), "K1 jobs");
      if (err.empty()) ck(upload(&dk2, k2), "K2 jobs");
      if (err.empty()) ck(upload(&dk2t, k2t), "K2 tasks");
      Profiler off;
      if (err.empty())
        for (const Chunk& c : chunks) launch_heff_fp64(s_, q, q, src, dst, T, dk1, dk2, dk2t, c, 0, &off);
      if (err.empty()) ck(cudaGetLastError(), "launch");
    }
    const auto cp = pieces_of(st.copies);
    if (err.empty() && !cp.empty() && ck(upload(&dcp, cp), "copies") && ck(upload(&dct, st.copy_terms), "copy terms"))
      group_kernel<<<unsigned(cp.size()), 256, 0, s_>>>(dcp, dct, src, dst);
    if (err.empty()) ck(cudaGetLastError(), "launch");
    if (err.empty()) ck(cudaStreamSynchronize(s_), "step");
    void* ps[] = {src, q, T, did, dtp, dcp, dtt, dct, dk1, dk2, dk2t};
    for (void* p : ps) cudaFree(p);
    if (!err.empty()) {
      cudaFree(dst);
      return err;
    }
    *out = dst;
    return "";
  }

 private:
  int device_;
  cudaStream_t s_;
  int64_t budget_;
  double* cur_ = nullptr;
  int64_t size_ = 0;
};

class HostBackend : public RenormBackend {
 public:
  int64_t size() const override { return int64_t(cur_.size()); }
  std::vector<double> take_host() override { return std::move(cur_); }
  std::string run(const RStep& st) override {
    std::vector<double> src(size_t(std::max<int64_t>(st.src_size, 1)), 0.0);
    std::copy(cur_.begin(), cur_.begin() + st.old_size, src.begin());
    for (const RIdent& r : st.idents)
      for (int i = 0; i < r.d; ++i) src[size_t(r.off + int64_t(i) * (r.d + 1))] = r.c;
    for (const RGroup& g : st.temps)
      for (int t = g.t0; t < g.t1; ++t) {
        const RTerm& x = st.temp_terms[t];
        for (int64_t i = 0; i < g.n; ++i) src[size_t(g.dst + i)] += x.w * src[size_t(x.src + i)];
      }
    cur_.assign(size_t(std::max<int64_t>(st.dst_size, 1)), 0.0);
    std::vector<double> T;
    for (const RTask& t : st.tasks) {
      // T = E D^T (k1 x n), then F += v A T
      T.assign(size_t(t.k1) * t.n, 0.0);
      const double* E = &src[size_t(t.e)];
      const double* D = &st.q[size_t(t.d)];
      const double* A = &st.q[size_t(t.a)];
      for (int kk = 0; kk < t.k2; ++kk)
        for (int c = 0; c < t.n; ++c) {
          const double dv = D[c + int64_t(kk) * t.n];
          if (dv == 0.0) continue;
          for (int r = 0; r < t.k1; ++r) T[r + size_t(c) * t.k1] += E[r + int64_t(kk) * t.k1] * dv;
        }
      double* F = &cur_[size_t(t.f)];
      for (int c = 0; c < t.n; ++c)
        for (int kk = 0; kk < t.k1; ++kk) {
          const double tv = t.v * T[kk + size_t(c) * t.k1];
          if (tv == 0.0) continue;
          for (int r = 0; r < t.m; ++r) F[r + int64_t(c) * t.m] += A[r + int64_t(kk) * t.m] * tv;
        }
      flops += 2.0 * (double(t.k1) * t.k2 * t.n + double(t.m) * t.k1 * t.n);
    }
    for (const RGroup& g : st.copies)
      for (int t = g.t0; t < g.t1; ++t) {
        const RTerm& x = st.copy_terms[t];
        for (int64_t i = 0; i < g.n; ++i) cur_[size_t(g.dst + i)] += x.w * src[size_t(x.src + i)];
      }
    if (st.dst_size == 0) cur_.clear();
    return "";
  }

 private:
  std::vector<double> cur_;
};

}  // namespace

RenormBackend* make_host_backend() { return new HostBackend(); }
RenormBackend* make_device_backend(int device, void* stream, int64_t t_budget_bytes) {
  return new DeviceBackend(device, stream, t_budget_bytes);
}

}  // namespace su2
