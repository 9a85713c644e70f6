// Renormalisation work of the ab initio environment (Sec. II.C, Sec. IV.D):
// one step turns the operators of a block into those of the block grown by
// one orbital.  The host plans a step as lists of plain array operations;
// a backend (host loops or the GPU) executes them.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace su2 {

// F(m x n) += v * A(m x k1) * E(k1 x k2) * D(n x k2)^T, column-major,
// contiguous: F in the destination arena, A and D in the Q arena (blocks of
// the transposed MPS tensors), E in the source arena.
struct RTask {
  int64_t f, a, e, d;
  int32_t m, k1, k2, n;
  double v;
};

// dst[i] += sum_j w_j * src_j[i], i < n: one destination range and its terms.
struct RGroup {
  int64_t dst, n;
  int32_t t0, t1;  // terms [t0, t1) of RStep::terms
};
struct RTerm {
  int64_t src;
  double w;
};

// src[off + i * (d + 1)] = c for i < d: an identity block written into the
// (zeroed) part of the source arena.
struct RIdent {
  int64_t off;
  int32_t d;
  double c;
};

struct RStep {
  int64_t old_size = 0;        // doubles of the current arena, copied to [0, old_size) of the source arena
  int64_t src_size = 0;        // source arena: the old operators, then identities and temporaries (zeroed)
  std::vector<RIdent> idents;  // written first
  std::vector<RGroup> temps;   // then these sums inside the source arena (temporaries from old operators)
  std::vector<RTerm> temp_terms;
  std::vector<double> q;       // the Q arena
  int64_t dst_size = 0;        // destination arena (zeroed), the next current arena
  std::vector<RTask> tasks;    // products into the destination
  std::vector<RGroup> copies;  // then these sums from the source into the destination
  std::vector<RTerm> copy_terms;
};

class RenormBackend {
 public:
  virtual ~RenormBackend() {}
  // executes a step: the destination arena becomes the current arena
  virtual std::string run(const RStep& st) = 0;
  // executes a step on an explicit old arena (device), which is kept; the
  // destination arena is returned (the caller owns it; device backend only)
  virtual std::string run_keep(const RStep& st, const double* old, double** out) {
    (void)st;
    (void)old;
    *out = nullptr;
    return "renormalisation on an explicit arena needs a device context";
  }
  virtual int64_t size() const = 0;
  // hands the current arena over (host vector or device pointer)
  virtual std::vector<double> take_host() { return {}; }
  virtual double* take_device() { return nullptr; }
  double flops = 0.0;  // of the products executed (2 (k1 k2 n + m k1 n) per task)
};

RenormBackend* make_host_backend();
RenormBackend* make_device_backend(int device, void* stream, int64_t t_budget_bytes);

}  // namespace su2
