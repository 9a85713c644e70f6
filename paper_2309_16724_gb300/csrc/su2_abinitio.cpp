// Ab initio environment: the Hamiltonian of Eq. 1 from one- and two-electron
// integrals, in the spin-adapted normal/complementary partition of Sec. II.A,
// with block operators renormalised from a seeded SU(2) MPS one orbital at a
// time (block x site with the W9j^(l) factor on the left, site x block with
// W9j^(r) on the right, Sec. II.C), and the operator-table of Eq. 2 at the
// two-site bond.
//
// * H = sum h_ij sum_s c+_is c_js + 1/2 sum (ij|kl) sum_st c+_is c+_kt c_lt c_js
//   is a sum of "strings": ordered products of rank-1/2 tensors a+_i
//   (components c+_{i,up}, c+_{i,dn}) and a~_i (components c_{i,dn},
//   -c_{i,up}) in Jordan-Wigner order (orbital, creators first), each with
//   a table of coefficients over the spin components.
// * A coupled product is a tree of Clebsch-Gordan couplings; coefficients
//   of a string in a coupled basis, and recoupling coefficients between
//   two trees, are inner products of component tables (the coupled bases
//   are orthonormal).
// * Right block: complementary operators C(O) for every set O of at most two
//   elementary operators outside the block (H_R for O empty), defined by
//   H = sum_O [O x C(O)]^0; a block grown by orbital s gets
//   C'(O') = sum_Y W [Y x C(O' + Y)] over strings Y on s.  Left block:
//   normal operators with one and two factors, C_L(O) for |O| <= 1.
// * Middle bond: each string belongs to exactly one family of rows, so
//   that the rows of Eq. 2 sum to H.
// The numerics of every step (products Q^T [Y x X] Q and sums of blocks)
// run on the GPU through the grouped FP64 kernels (su2_renorm.h), or on the
// host for a host-only context.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "su2_internal.h"
#include "su2_renorm.h"

namespace su2 {
namespace {

double cgc(int j1, int m1, int j2, int m2, int J, int M) { return cg_coef(j1, m1, j2, m2, J, M); }

// ------------------------------------------------------------------ coupling trees
// signatures: "e" (rank 1/2, two components), "0" (scalar), "x<j>" (rank
// j/2), "(<left>,<right>)<K>"; the component table of a tree over its
// non-scalar leaves, row-major in leaf order
struct TreeVal {
  int j = 0;
  std::map<int, std::vector<double>> comp;  // total component M -> table
};

std::string node(const std::string& a, const std::string& b, int K) {
  return "(" + a + "," + b + ")" + std::to_string(K);
}
std::string xleaf(int j) { return "x" + std::to_string(j); }
std::string lnest(int n, const std::vector<int>& lab) {
  if (n == 0) return "0";
  std::string t = "e";
  for (int i = 1; i < n; ++i) t = node(t, "e", lab[i - 1]);
  return t;
}

class Trees {
 public:
  const TreeVal& get(const std::string& s) {
    auto it = memo_.find(s);
    if (it != memo_.end()) return it->second;
    size_t pos = 0;
    TreeVal v = parse(s, pos);
    return memo_.emplace(s, std::move(v)).first->second;
  }
  double overlap(const std::string& a, const std::string& b) {
    const std::string key = a + "|" + b;
    auto it = ov_.find(key);
    if (it != ov_.end()) return it->second;
    const TreeVal& x = get(a);
    const TreeVal& y = get(b);
    double r = 0.0;
    auto ix = x.comp.find(0), iy = y.comp.find(0);
    if (ix != x.comp.end() && iy != y.comp.end()) {
      if (ix->second.size() != iy->second.size()) throw std::runtime_error("overlap of trees over different leaves");
      for (size_t i = 0; i < ix->second.size(); ++i) r += ix->second[i] * iy->second[i];
    }
    ov_[key] = r;
    return r;
  }
  // coefficient of a string's component table on a rank-0 tree
  double coef(const std::string& t, const double* F, int nF) {
    const TreeVal& x = get(t);
    auto ix = x.comp.find(0);
    if (ix == x.comp.end()) return 0.0;
    if (int(ix->second.size()) != nF) throw std::runtime_error("string and tree differ in their leaves");
    double r = 0.0;
    for (int i = 0; i < nF; ++i) r += ix->second[i] * F[i];
    return r;
  }

 private:
  TreeVal parse(const std::string& s, size_t& pos) {
    TreeVal v;
    const char c = s[pos];
    if (c == 'e') {
      ++pos;
      v.j = 1;
      v.comp[1] = {1.0, 0.0};
      v.comp[-1] = {0.0, 1.0};
      return v;
    }
    if (c == '0') {
      ++pos;
      v.j = 0;
      v.comp[0] = {1.0};
      return v;
    }
    if (c == 'x') {
      ++pos;
      int j = 0;
      while (pos < s.size() && std::isdigit((unsigned char)s[pos])) j = 10 * j + (s[pos++] - '0');
      v.j = j;
      for (int idx = 0, m = j; m >= -j; m -= 2, ++idx) {
        std::vector<double> e(size_t(j + 1), 0.0);
        e[size_t(idx)] = 1.0;
        v.comp[m] = e;
      }
      return v;
    }
    // "(" left "," right ")" K
    ++pos;
    TreeVal l = parse(s, pos);
    ++pos;  // ','
    TreeVal r = parse(s, pos);
    ++pos;  // ')'
    int K = 0;
    while (pos < s.size() && std::isdigit((unsigned char)s[pos])) K = 10 * K + (s[pos++] - '0');
    v.j = K;
    for (auto& [ml, vl] : l.comp)
      for (auto& [mr, vr] : r.comp) {
        const int M = ml + mr;
        if (std::abs(M) > K) continue;
        const double cgv = cgc(l.j, ml, r.j, mr, K, M);
        if (cgv == 0.0) continue;
        std::vector<double>& out = v.comp[M];
        if (out.empty()) out.assign(vl.size() * vr.size(), 0.0);
        for (size_t a = 0; a < vl.size(); ++a)
          for (size_t b = 0; b < vr.size(); ++b) out[a * vr.size() + b] += cgv * vl[a] * vr[b];
      }
    return v;
  }
  std::unordered_map<std::string, TreeVal> memo_;
  std::unordered_map<std::string, double> ov_;
};

std::vector<std::vector<int>> labelings(int n) {
  std::vector<std::vector<int>> res;
  if (n <= 1) {
    res.push_back({});
    return res;
  }
  for (const auto& lab : labelings(n - 1)) {
    const int j = lab.empty() ? 1 : lab.back();
    for (int K = std::abs(j - 1); K <= j + 1; K += 2) {
      auto x = lab;
      x.push_back(K);
      res.push_back(x);
    }
  }
  return res;
}
int lab_rank(int n, const std::vector<int>& lab) { return n == 0 ? 0 : (n == 1 ? 1 : lab.back()); }

// ------------------------------------------------------------------ strings
struct EOp {
  int orb, dag;  // dag 1: a+, 0: a~
  bool operator==(const EOp& o) const { return orb == o.orb && dag == o.dag; }
};
int code(const EOp& o) { return 2 * o.orb + (1 - o.dag); }  // Jordan-Wigner order: ascending code
using Str = std::vector<EOp>;

uint64_t skey(const Str& s) {
  uint64_t k = uint64_t(s.size());
  for (const EOp& o : s) k = (k << 14) | uint64_t(code(o));
  return k;
}

// two equal elementary operators coupled directly to rank 1 vanish
bool valid(const Str& o, const std::vector<int>& lab) { return !(o.size() >= 2 && o[0] == o[1] && lab[0] == 2); }

struct Table16 {
  int n = 0;
  double v[16] = {0};
};

class Strings {
 public:
  Strings(int L, const double* h, const double* eri) {
    // sum_s c+_s c_s and sum_st c+_s c+_t c_t c_s over the components of the
    // tensors; c_up = -a~_{-1/2} (component 1), c_dn = a~_{+1/2} (component 0)
    auto cs = [](int s) { return s == 0 ? -1.0 : 1.0; };
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j) {
        const double x = h[size_t(i) * L + j];
        if (x == 0.0) continue;
        double F[4] = {0};
        for (int s = 0; s < 2; ++s) F[s * 2 + (1 - s)] = x * cs(s);
        add({{i, 1}, {j, 0}}, F);
      }
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j)
        for (int k = 0; k < L; ++k)
          for (int l = 0; l < L; ++l) {
            const double x = eri[((size_t(i) * L + j) * L + k) * L + l];
            if (x == 0.0) continue;
            double F[16] = {0};
            for (int s = 0; s < 2; ++s)
              for (int t = 0; t < 2; ++t) F[s * 8 + t * 4 + (1 - t) * 2 + (1 - s)] = 0.5 * x * cs(s) * cs(t);
            add({{i, 1}, {k, 1}, {l, 0}, {j, 0}}, F);
          }
  }
  const Table16* find(const Str& s) const {
    auto it = map_.find(skey(s));
    return it == map_.end() ? nullptr : &it->second;
  }

 private:
  void add(const Str& ops, const double* F) {
    const int n = int(ops.size());
    std::vector<int> ord(static_cast<size_t>(n));
    for (int a = 0; a < n; ++a) ord[a] = a;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return code(ops[a]) < code(ops[b]); });
    // sign of the permutation (every swap is between different orbitals)
    int inv = 0;
    for (int a = 0; a < n; ++a)
      for (int b = a + 1; b < n; ++b)
        if (ord[a] > ord[b]) ++inv;
    Str sorted(static_cast<size_t>(n));
    for (int a = 0; a < n; ++a) sorted[a] = ops[ord[a]];
    Table16& t = map_[skey(sorted)];
    t.n = n;
    const int N = 1 << n;
    for (int idx = 0; idx < N; ++idx) {
      // component of new position a is bit (n-1-a) of idx; it is old operator ord[a]
      int old = 0;
      for (int a = 0; a < n; ++a)
        if ((idx >> (n - 1 - a)) & 1) old |= 1 << (n - 1 - ord[a]);
      t.v[idx] += (inv % 2 ? -1.0 : 1.0) * F[old];
    }
  }
  std::unordered_map<uint64_t, Table16> map_;
};

// ------------------------------------------------------------------ site operators
// reduced 3x3 matrix (CG form) of a coupled product of tensors on one orbital
// from its component matrices on the four states |0>, |up>, |dn>, |2> = c+_up c+_dn |0>
bool site_red(Trees& tr, const std::vector<int>& dags, const std::vector<int>& lab, SiteOp& out) {
  const int n = int(dags.size());
  out = SiteOp();
  out.n = 3;
  if (n == 0) {
    out.red[0][0] = out.red[1][1] = out.red[2][2] = 1.0;
    return true;
  }
  double cu[4][4] = {{0}}, cd[4][4] = {{0}};
  cu[1][0] = 1.0;
  cu[3][2] = 1.0;
  cd[2][0] = 1.0;
  cd[3][1] = -1.0;
  auto elem = [&](int dag, int comp, double M[4][4]) {
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        if (dag) M[r][c] = comp == 0 ? cu[r][c] : cd[r][c];
        else M[r][c] = comp == 0 ? cd[c][r] : -cu[c][r];  // a~_{+1/2} = c_dn, a~_{-1/2} = -c_up
      }
  };
  const TreeVal& t = tr.get(lnest(n, lab));
  const int k = t.j;
  std::map<int, std::array<std::array<double, 4>, 4>> T;
  for (auto& [q, tab] : t.comp) {
    std::array<std::array<double, 4>, 4> acc{};
    for (size_t idx = 0; idx < tab.size(); ++idx) {
      if (tab[idx] == 0.0) continue;
      double P[4][4] = {{0}};
      for (int i = 0; i < 4; ++i) P[i][i] = 1.0;
      for (int a = 0; a < n; ++a) {
        double Mx[4][4], R[4][4] = {{0}};
        elem(dags[a], int((idx >> (n - 1 - a)) & 1), Mx);
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j)
            for (int l = 0; l < 4; ++l) R[i][j] += P[i][l] * Mx[l][j];
        std::memcpy(P, R, sizeof(P));
      }
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] += tab[idx] * P[i][j];
    }
    T[q] = acc;
  }
  // site multiplets: (N, 2S, [(2m, state)])
  struct St { int twoS; int nm; int m[2]; int f[2]; };
  const St st[3] = {{0, 1, {0, 0}, {0, 0}}, {1, 2, {1, -1}, {1, 2}}, {0, 1, {0, 0}, {3, 3}}};
  bool nz = false;
  for (int so = 0; so < 3; ++so)
    for (int si = 0; si < 3; ++si) {
      bool have = false;
      double val = 0.0;
      for (int a = 0; a < st[so].nm && !have; ++a)
        for (int b = 0; b < st[si].nm && !have; ++b) {
          const int q = st[so].m[a] - st[si].m[b];
          if (std::abs(q) > k || !T.count(q)) continue;
          const double c = cgc(st[si].twoS, st[si].m[b], k, q, st[so].twoS, st[so].m[a]);
          if (c == 0.0) continue;
          val = T[q][st[so].f[a]][st[si].f[b]] / c;
          have = true;
        }
      if (have && std::abs(val) > 1e-15) {
        out.red[so][si] = val;
        nz = true;
      }
    }
  int dN = 0;
  for (int d : dags) dN += d ? 1 : -1;
  out.k = k;
  out.dN = dN;
  out.parity = n % 2;
  return nz;
}

// ------------------------------------------------------------------ blocks
struct OpDir {
  int k = 0, dN = 0, par = 0;
  std::vector<std::pair<int32_t, int64_t>> blk;  // (qo * 4096 + qi, offset), sorted
  int64_t find(int qo, int qi) const {
    const int32_t key = qo * 4096 + qi;
    auto it = std::lower_bound(blk.begin(), blk.end(), std::make_pair(key, int64_t(-1)));
    return (it != blk.end() && it->first == key) ? it->second : -1;
  }
};

// an arena layout: operators with their allowed blocks
struct Layout {
  std::vector<Sector> sec;
  std::vector<OpDir> ops;
  std::map<std::string, int> index;
  int64_t size = 0;
  int add(const std::string& key, int k, int dN, int par) {
    OpDir d;
    d.k = k;
    d.dN = dN;
    d.par = par;
    for (int qo = 0; qo < int(sec.size()); ++qo)
      for (int qi = 0; qi < int(sec.size()); ++qi)
        if (sec[qo].N == sec[qi].N + dN && triangle(sec[qi].twoS, k, sec[qo].twoS)) {
          d.blk.emplace_back(qo * 4096 + qi, size);
          size += (int64_t(sec[qo].dim) * sec[qi].dim + 1) & ~int64_t(1);
        }
    std::sort(d.blk.begin(), d.blk.end());
    ops.push_back(d);
    index[key] = int(ops.size()) - 1;
    return int(ops.size()) - 1;
  }
  int find(const std::string& key) const {
    auto it = index.find(key);
    return it == index.end() ? -1 : it->second;
  }
};

std::string opkey(char kind, const Str& o, const std::vector<int>& lab) {
  std::string s(1, kind);
  for (const EOp& x : o) s += ":" + std::to_string(x.orb) + (x.dag ? "+" : "~");
  s += "|";
  for (int l : lab) s += std::to_string(l) + ",";
  return s;
}

// an operator source of a step: an operator of the old block, a multiple of
// the identity, or a temporary (a sum of old operators) in the source arena
struct Src {
  enum { NONE, OLD, IDENT, TEMP } kind = NONE;
  int idx = -1;     // operator in the old layout or the temporary layout
  double c = 1.0;   // IDENT: the multiple
  int k = 0, par = 0;
};

struct Contrib {
  double coef;
  SiteOp Y;
  Src X;
  int K;
};

struct Stack {
  int qp, s, r0, d;
};

class Builder {
 public:
  Builder(const su2_hamiltonian& H, int device, void* stream, int64_t budget)
      : H_(H), L_(H.n_left + 2 + H.n_right), strings_(L_, H.h, H.eri), device_(device), stream_(stream),
        budget_(budget) {
    site_states(SU2_SITE_ORBITAL, sN_, sS_);
  }

  // the operators of one block after its last step; `left` selects the side
  struct Side {
    Layout lay;
    std::unique_ptr<RenormBackend> own;
    RenormBackend* be = nullptr;
    std::vector<int> orbs;
    const double* arena = nullptr;  // keep mode: the block's device arena (not consumed)
    int64_t arena_size = 0;
  };

  // the caller's MPS tensors of one step (the layout of su2_hamiltonian's
  // mps_left / mps_right), read from *pos onwards
  std::vector<std::vector<double>> step_tensors(const std::vector<Sector>& prev, const std::vector<Sector>& cur,
                                                const double* mps, size_t* pos) const {
    std::vector<std::vector<double>> Q(cur.size());
    for (size_t qo = 0; qo < cur.size(); ++qo) {
      int64_t r0 = 0;
      for (const Sector& p : prev)
        for (int si = 0; si < 3; ++si)
          if (p.N + sN_[si] == cur[qo].N && triangle(p.twoS, sS_[si], cur[qo].twoS)) r0 += p.dim;
      const size_t n = size_t(r0) * size_t(cur[qo].dim);
      Q[qo].assign(mps + *pos, mps + *pos + n);
      *pos += n;
    }
    return Q;
  }

  // the seeded MPS tensor of sector qo at growth step `step` (side 2: left,
  // 3: right): the Q factor of a counter-generated r0 x d matrix
  std::vector<double> seeded_tensor(uint64_t side, int step, int qo, int r0, int d) const {
    return seeded_mps_tensor(H_.seed, side, step, qo, r0, d);
  }

  // the seeded MPS tensors of one step (per new sector, stacked rows x dim)
  std::vector<std::vector<double>> seeded_tensors(bool left, int step, const std::vector<Sector>& prev,
                                                  const std::vector<Sector>& cur) const {
    std::vector<std::vector<double>> Q(cur.size());
    for (size_t qo = 0; qo < cur.size(); ++qo) {
      int r0 = 0;
      for (const Sector& p : prev)
        for (int si = 0; si < 3; ++si)
          if (p.N + sN_[si] == cur[qo].N && triangle(p.twoS, sS_[si], cur[qo].twoS)) r0 += p.dim;
      if (r0 < cur[qo].dim) return {};
      Q[qo] = seeded_tensor(left ? 2 : 3, step, int(qo), r0, cur[qo].dim);
    }
    return Q;
  }

  std::string grow(bool left, const std::vector<std::vector<Sector>>& chain, Side& out, const double* mps = nullptr) {
    out.own.reset(device_ >= 0 ? make_device_backend(device_, stream_, budget_) : make_host_backend());
    out.be = out.own.get();
    Layout old;
    old.sec = chain[0];
    std::vector<int> orbs;
    size_t pos = 0;
    for (size_t step = 1; step < chain.size(); ++step) {
      const int s = left ? int(step) - 1 : L_ - int(step);
      std::vector<std::vector<double>> Q;
      if (mps) Q = step_tensors(chain[step - 1], chain[step], mps, &pos);
      std::string err = step_block(left, int(step), s, chain[step - 1], chain[step], mps ? &Q : nullptr, orbs, old,
                                   *out.be, nullptr, 0, nullptr);
      if (!err.empty()) return err;
      if (left) orbs.push_back(s);
      else orbs.insert(orbs.begin(), s);
    }
    out.lay = old;
    out.orbs = orbs;
    return "";
  }

  std::string assemble(OpTable& table, SideOps& Lops, SideOps& Rops, double* flops);

  // ---------------------------------------------------------------- one step
  // Grows a block by orbital s: the new bond `cur` and the MPS tensor Qin
  // (per new sector, its stacked rows x dim, column-major), or the seeded
  // tensor of `step` when Qin is null.  Keep mode (keep_out non-null): the
  // old arena keep_old of keep_size doubles is read and kept, the new arena
  // returned; otherwise the backend's current arena is replaced.
  std::string step_block(bool left, int step, int s, const std::vector<Sector>& prev, const std::vector<Sector>& cur,
                         const std::vector<std::vector<double>>* Qin, const std::vector<int>& orbs, Layout& old,
                         RenormBackend& be, const double* keep_old, int64_t keep_size, double** keep_out) {
    RStep st;
    st.old_size = keep_out ? keep_size : be.size();
    old_ = &old;
    orbs_ = &orbs;
    left_ = left;
    prevsec_ = &prev;
    // source arena: old operators, identities of the previous bond, temporaries
    int64_t off = st.old_size;
    ident_.assign(prev.size(), -1);
    for (size_t q = 0; q < prev.size(); ++q) {
      ident_[q] = off;
      st.idents.push_back(RIdent{off, prev[q].dim, 1.0});
      off += (int64_t(prev[q].dim) * prev[q].dim + 1) & ~int64_t(1);
    }
    temps_ = Layout();
    temps_.sec = prev;
    temp_base_ = off;
    temp_groups_.clear();
    temp_terms_.clear();
    // MPS tensor of the step: stacked rows (previous sector, site state) per new sector, Q
    const uint64_t side = left ? 2 : 3;
    std::vector<std::vector<Stack>> stacks(cur.size());
    std::vector<int64_t> qoff(cur.size());
    for (int qo = 0; qo < int(cur.size()); ++qo) {
      int r0 = 0;
      for (int qp = 0; qp < int(prev.size()); ++qp)
        for (int si = 0; si < 3; ++si)
          if (prev[qp].N + sN_[si] == cur[qo].N && triangle(prev[qp].twoS, sS_[si], cur[qo].twoS)) {
            stacks[qo].push_back(Stack{qp, si, r0, prev[qp].dim});
            r0 += prev[qp].dim;
          }
      const int d = cur[qo].dim;
      if (r0 < d) return "bond dimension exceeds the states available from the previous bond";
      std::vector<double> G(size_t(r0) * d);
      if (Qin) {
        if ((*Qin)[size_t(qo)].size() != G.size()) return "MPS tensor does not match the stacked rows of its sector";
        G = (*Qin)[size_t(qo)];
      } else {
        G = seeded_tensor(side, step, qo, r0, d);
      }
      qoff[qo] = int64_t(st.q.size());
      // Q^T (d x r0), column-major
      st.q.resize(st.q.size() + size_t(r0) * d);
      double* qt = &st.q[size_t(qoff[qo])];
      for (int c = 0; c < r0; ++c)
        for (int r = 0; r < d; ++r) qt[r + size_t(c) * d] = G[size_t(c) + size_t(r) * r0];
    }
    // the new operators and their contributions
    Layout nl;
    nl.sec = cur;
    std::vector<std::vector<Contrib>> contribs;
    auto add_op = [&](const std::string& key, int k, int dN, int par, std::vector<Contrib>&& cs) {
      if (cs.empty()) return;
      nl.add(key, k, dN, par);
      contribs.push_back(std::move(cs));
    };
    SiteOp Isite;
    site_red(tr_, {}, {}, Isite);
    std::vector<int> new_orbs = orbs;
    if (left) new_orbs.push_back(s);
    else new_orbs.insert(new_orbs.begin(), s);
    // elementary operators of the new block
    for (int o : new_orbs)
      for (int dag = 1; dag >= 0; --dag) {
        const Str x{{o, dag}};
        std::vector<Contrib> cs;
        if (o == s) {
          SiteOp Y;
          site_red(tr_, {dag}, {}, Y);
          cs.push_back(Contrib{1.0, Y, ident(1.0), 1});
        } else {
          cs.push_back(Contrib{1.0, Isite, old_src(opkey('N', x, {})), 1});
        }
        add_op(opkey('N', x, {}), 1, dag ? 1 : -1, 1, std::move(cs));
      }
    if (left) {
      // normal operators with two factors
      std::vector<EOp> el;
      for (int o : new_orbs) {
        el.push_back({o, 1});
        el.push_back({o, 0});
      }
      for (size_t a = 0; a < el.size(); ++a)
        for (size_t b = a; b < el.size(); ++b) {
          const Str pr{el[a], el[b]};
          for (const auto& lab : labelings(2)) {
            if (!valid(pr, lab)) continue;
            std::vector<Contrib> cs;
            const int K = lab[0];
            if (pr[0].orb != s && pr[1].orb != s) {
              cs.push_back(Contrib{1.0, Isite, old_src(opkey('P', pr, lab)), K});
            } else if (pr[0].orb != s) {
              SiteOp Y;
              site_red(tr_, {pr[1].dag}, {}, Y);
              cs.push_back(Contrib{1.0, Y, old_src(opkey('N', Str{pr[0]}, {})), K});
            } else {
              SiteOp Y;
              if (!site_red(tr_, {pr[0].dag, pr[1].dag}, lab, Y)) continue;
              cs.push_back(Contrib{1.0, Y, ident(1.0), K});
            }
            const int dN = (pr[0].dag ? 1 : -1) + (pr[1].dag ? 1 : -1);
            add_op(opkey('P', pr, lab), K, dN, 0, std::move(cs));
          }
        }
    }
    // complementary operators over the outside elementary operators
    std::vector<EOp> outside;
    if (left) {
      for (int o = s + 1; o < L_; ++o) {
        outside.push_back({o, 1});
        outside.push_back({o, 0});
      }
    } else {
      for (int o = 0; o < s; ++o) {
        outside.push_back({o, 1});
        outside.push_back({o, 0});
      }
    }
    const int maxO = left ? 1 : 2;
    std::vector<std::pair<Str, std::vector<int>>> keys;
    keys.push_back({{}, {}});
    for (const EOp& o : outside) keys.push_back({{o}, {}});
    if (maxO >= 2)
      for (size_t a = 0; a < outside.size(); ++a)
        for (size_t b = a; b < outside.size(); ++b) {
          const Str pr{outside[a], outside[b]};
          for (const auto& lab : labelings(2))
            if (valid(pr, lab)) keys.push_back({pr, lab});
        }
    for (const auto& [O1, lam1] : keys) {
      const int n1 = int(O1.size());
      const int k1 = lab_rank(n1, lam1);
      int dN = 0;
      for (const EOp& x : O1) dN += x.dag ? 1 : -1;
      std::vector<Contrib> cs = recursion(O1, lam1, s);
      add_op(opkey('C', O1, lam1), k1, -dN, n1 % 2, std::move(cs));
    }
    // temporaries into the source arena
    st.src_size = temp_base_ + temps_.size;
    for (auto& g : temp_groups_) g.dst += temp_base_;
    st.temps = temp_groups_;
    st.temp_terms = temp_terms_;
    // products into the destination arena
    st.dst_size = nl.size;
    for (size_t oi = 0; oi < nl.ops.size(); ++oi) {
      const OpDir& od = nl.ops[oi];
      for (const auto& [key, foff] : od.blk) {
        const int qo = key / 4096, qi = key % 4096;
        for (const Contrib& c : contribs[oi]) {
          const OpDir* xd = c.X.kind == Src::OLD ? &old.ops[c.X.idx] : (c.X.kind == Src::TEMP ? &temps_.ops[c.X.idx] : nullptr);
          for (const Stack& ro : stacks[qo])
            for (const Stack& ri : stacks[qi]) {
              const double y = c.Y.red[ro.s][ri.s];
              if (y == 0.0) continue;
              int64_t eoff;
              if (c.X.kind == Src::IDENT) {
                if (ro.qp != ri.qp) continue;
                eoff = ident_[ro.qp];
              } else {
                eoff = xd->find(ro.qp, ri.qp);
                if (eoff < 0) continue;
                if (c.X.kind == Src::TEMP) eoff += temp_base_;
              }
              double ct, sg;
              if (left) {
                ct = ctilde(prev[ri.qp].twoS, sS_[ri.s], cur[qi].twoS, c.X.k, c.Y.k, c.K, prev[ro.qp].twoS, sS_[ro.s],
                            cur[qo].twoS);
                sg = (c.Y.parity && (prev[ri.qp].N % 2)) ? -1.0 : 1.0;
              } else {
                ct = ctilde(sS_[ri.s], prev[ri.qp].twoS, cur[qi].twoS, c.Y.k, c.X.k, c.K, sS_[ro.s], prev[ro.qp].twoS,
                            cur[qo].twoS);
                sg = (c.X.par && (sN_[ri.s] % 2)) ? -1.0 : 1.0;
              }
              if (ct == 0.0) continue;
              const double v = c.coef * y * ct * sg * (c.X.kind == Src::IDENT ? c.X.c : 1.0);
              st.tasks.push_back(RTask{foff, qoff[qo] + int64_t(ro.r0) * cur[qo].dim, eoff,
                                       qoff[qi] + int64_t(ri.r0) * cur[qi].dim, cur[qo].dim, prev[ro.qp].dim,
                                       prev[ri.qp].dim, cur[qi].dim, v});
            }
        }
      }
    }
    std::string err = keep_out ? be.run_keep(st, keep_old, keep_out) : be.run(st);
    if (!err.empty()) return err;
    old = nl;
    return "";
  }

 private:

  Src ident(double c) {
    Src x;
    x.kind = Src::IDENT;
    x.c = c;
    return x;
  }
  Src old_src(const std::string& key) {
    Src x;
    const int i = old_->find(key);
    if (i < 0) return x;
    x.kind = Src::OLD;
    x.idx = i;
    x.k = old_->ops[i].k;
    x.par = old_->ops[i].par;
    return x;
  }

  // C(O, lam) of the old block: stored, a number times the identity, or a
  // temporary sum of the old block's normal operators
  Src get(const Str& O, const std::vector<int>& lam) {
    const int n = int(O.size());
    const bool empty = orbs_->empty();
    const int stored = left_ ? 1 : 2;
    if (n <= stored && !empty) return old_src(opkey('C', O, lam));
    const int kO = lab_rank(n, lam);
    const std::string tkey = opkey('T', O, lam);
    int ti = temps_.find(tkey);
    if (ti >= 0) {
      Src x;
      x.kind = Src::TEMP;
      x.idx = ti;
      x.k = temps_.ops[ti].k;
      x.par = temps_.ops[ti].par;
      return x;
    }
    // terms of the sum
    std::vector<std::pair<Src, double>> terms;
    double scalar = 0.0;
    if (n % 2 == 0 && kO == 0) {
      if (const Table16* F = strings_.find(O)) scalar = tr_.coef(lnest(n, lam), F->v, 1 << n);
    }
    if (!empty) {
      std::vector<EOp> el;
      for (int o : *orbs_) {
        el.push_back({o, 1});
        el.push_back({o, 0});
      }
      if (n % 2 == 1 && kO == 1) {  // one block factor
        for (const EOp& x : el) {
          Str S = left_ ? Str{x} : O;
          if (left_) S.insert(S.end(), O.begin(), O.end());
          else S.push_back(x);
          const Table16* F = strings_.find(S);
          if (!F) continue;
          const std::string t = left_ ? node("e", lnest(n, lam), 0) : node(lnest(n, lam), "e", 0);
          const double c = tr_.coef(t, F->v, 1 << (n + 1));
          if (c != 0.0) terms.push_back({old_src(opkey('N', Str{x}, {})), c});
        }
      } else if (left_ && n == 2) {  // two block factors (left block)
        for (size_t a = 0; a < el.size(); ++a)
          for (size_t b = a; b < el.size(); ++b) {
            Str S{el[a], el[b]};
            const Str pr = S;
            S.insert(S.end(), O.begin(), O.end());
            const Table16* F = strings_.find(S);
            if (!F) continue;
            for (const auto& mu : labelings(2)) {
              if (!valid(pr, mu) || mu[0] != kO) continue;
              const double c = tr_.coef(node(lnest(2, mu), lnest(n, lam), 0), F->v, 16);
              if (c != 0.0) terms.push_back({old_src(opkey('P', pr, mu)), c});
            }
          }
      }
    }
    if (terms.empty()) {
      if (scalar == 0.0) return Src();
      return ident(scalar);
    }
    // a temporary: its blocks are sums of the terms' blocks (and the identity)
    int dN = 0;
    for (const EOp& x : O) dN += x.dag ? 1 : -1;
    ti = temps_.add(tkey, kO, -dN, n % 2);
    const OpDir& td = temps_.ops[ti];
    for (const auto& [key, off] : td.blk) {
      const int qo = key / 4096, qi = key % 4096;
      const int64_t nel = int64_t((*prevsec_)[qo].dim) * (*prevsec_)[qi].dim;
      const int32_t t0 = int32_t(temp_terms_.size());
      for (const auto& [src, w] : terms) {
        if (src.kind != Src::OLD) continue;
        const int64_t so = old_->ops[src.idx].find(qo, qi);
        if (so >= 0) temp_terms_.push_back(RTerm{so, w});
      }
      if (scalar != 0.0 && qo == qi) temp_terms_.push_back(RTerm{ident_[qo], scalar});
      temp_groups_.push_back(RGroup{off, nel, t0, int32_t(temp_terms_.size())});
    }
    Src x;
    x.kind = Src::TEMP;
    x.idx = ti;
    x.k = kO;
    x.par = n % 2;
    return x;
  }

  // contributions of C'(O1, lam1) of the grown block: W [Y x C(O)]  (right,
  // O = O1 + Y) or W [C(O) x Y] (left, O = Y + O1) over strings Y on s
  std::vector<Contrib> recursion(const Str& O1, const std::vector<int>& lam1, int s) {
    const int n1 = int(O1.size());
    const int k1 = lab_rank(n1, lam1);
    std::vector<Contrib> cs;
    for (int nc = 0; nc <= 2; ++nc)
      for (int na = 0; na <= 2; ++na) {
        const int nY = nc + na;
        if (n1 + nY > 4) continue;
        Str Y;
        std::vector<int> dags;
        for (int i = 0; i < nc; ++i) {
          Y.push_back({s, 1});
          dags.push_back(1);
        }
        for (int i = 0; i < na; ++i) {
          Y.push_back({s, 0});
          dags.push_back(0);
        }
        Str O = left_ ? Y : O1;
        if (left_) O.insert(O.end(), O1.begin(), O1.end());
        else O.insert(O.end(), Y.begin(), Y.end());
        for (const auto& nu : labelings(nY)) {
          if (nY && !valid(Y, nu)) continue;
          SiteOp Yop;
          if (!site_red(tr_, dags, nu, Yop)) continue;
          const int kY = lab_rank(nY, nu);
          for (const auto& lam : labelings(int(O.size()))) {
            if (O.size() && !valid(O, lam)) continue;
            const int kX = lab_rank(int(O.size()), lam);
            if (!triangle(kY, kX, k1)) continue;
            double W;
            if (left_)
              W = tr_.overlap(node(node(xleaf(kX), lnest(nY, nu), k1), lnest(n1, lam1), 0),
                              node(xleaf(kX), lnest(int(O.size()), lam), 0));
            else
              W = tr_.overlap(node(lnest(n1, lam1), node(lnest(nY, nu), xleaf(kX), k1), 0),
                              node(lnest(int(O.size()), lam), xleaf(kX), 0));
            if (std::abs(W) < 1e-14) continue;
            Src X = get(O, lam);
            if (X.kind == Src::NONE || X.k != kX) continue;
            cs.push_back(Contrib{W, Yop, X, k1});
          }
        }
      }
    return cs;
  }

  su2_hamiltonian H_;
  int L_;
  Strings strings_;
  Trees tr_;
  int device_;
  void* stream_;
  int64_t budget_;
  std::vector<int> sN_, sS_;
  // state of the step being planned
  Layout* old_ = nullptr;
  const std::vector<int>* orbs_ = nullptr;
  const std::vector<Sector>* prevsec_ = nullptr;
  bool left_ = false;
  std::vector<int64_t> ident_;
  Layout temps_;
  int64_t temp_base_ = 0;
  std::vector<RGroup> temp_groups_;
  std::vector<RTerm> temp_terms_;


 public:
  Side lside, rside;
};

// ---------------------------------------------------------------- middle bond
// the final arena of one side: operators referenced by the table, copied (or
// summed) from the block's arena
struct Final {
  Layout lay;                          // final layout
  std::vector<RGroup> groups;          // copies into the final arena
  std::vector<RTerm> terms;
  std::vector<int64_t> ident;          // identity blocks in the source arena
  std::vector<RIdent> idents;
  int64_t src_size = 0;
  std::map<std::string, int> ids;      // table op id by key (0: identity)
  std::vector<BlockOp> descs;
};

// a final operator as sum_j w_j (source operator j); a source is an operator
// of the block layout (index) or, with idx = -1, the identity
struct Part {
  int idx;
  double w;
};

int final_op(Final& f, const Layout& src, const std::string& key, int k, int dN, int par,
             const std::vector<Part>& parts) {
  auto it = f.ids.find(key);
  if (it != f.ids.end()) return it->second;
  const int li = f.lay.add(key, k, dN, par);
  const OpDir& od = f.lay.ops[li];
  for (const auto& [bk, off] : od.blk) {
    const int qo = bk / 4096, qi = bk % 4096;
    const int32_t t0 = int32_t(f.terms.size());
    for (const Part& p : parts) {
      if (p.idx < 0) {
        if (qo == qi) f.terms.push_back(RTerm{f.ident[qo], p.w});
        continue;
      }
      const int64_t so = src.ops[p.idx].find(qo, qi);
      if (so >= 0) f.terms.push_back(RTerm{so, p.w});
    }
    f.groups.push_back(RGroup{off, int64_t(f.lay.sec[qo].dim) * f.lay.sec[qi].dim, t0, int32_t(f.terms.size())});
  }
  BlockOp d;
  d.name = key;
  d.k = k;
  d.dN = dN;
  d.parity = par;
  d.kind = OP_VALUES;
  f.descs.push_back(d);
  const int id = int(f.descs.size()) - 1;
  f.ids[key] = id;
  return id;
}

void init_final(Final& f, const std::vector<Sector>& sec, int64_t old_size) {
  f.lay.sec = sec;
  int64_t off = old_size;
  for (size_t q = 0; q < sec.size(); ++q) {
    f.ident.push_back(off);
    f.idents.push_back(RIdent{off, sec[q].dim, 1.0});
    off += (int64_t(sec[q].dim) * sec[q].dim + 1) & ~int64_t(1);
  }
  f.src_size = off;
  BlockOp I;
  I.name = "I";
  f.descs.push_back(I);
  f.ids["I"] = 0;
}

std::string Builder::assemble(OpTable& table, SideOps& Lops, SideOps& Rops, double* flops) {
  const int nL = int(lside.orbs.size()), p = nL, q = nL + 1;
  const Layout& LL = lside.lay;
  const Layout& RL = rside.lay;
  Final fl, fr;
  init_final(fl, LL.sec, lside.arena ? lside.arena_size : lside.be->size());
  init_final(fr, RL.sec, rside.arena ? rside.arena_size : rside.be->size());
  // the block Hamiltonians first (left / right operator 1)
  auto must = [](int i) {
    if (i < 0) throw std::runtime_error("missing block operator");
    return i;
  };
  const int iHL = LL.find(opkey('C', {}, {})), iHR = RL.find(opkey('C', {}, {}));
  if (iHL >= 0) final_op(fl, LL, "H", 0, 0, 0, {{iHL, 1.0}});
  if (iHR >= 0) final_op(fr, RL, "H", 0, 0, 0, {{iHR, 1.0}});
  SiteOp Isite;
  site_red(tr_, {}, {}, Isite);
  auto side_of = [&](int orb) { return orb < nL ? 0 : (orb == p ? 1 : (orb == q ? 2 : 3)); };
  struct Row {
    double a;
    int A, D, k;
    SiteOp B, C;
  };
  std::vector<Row> rows;
  // site operators of the parts on p and q with their labels
  auto site_variants = [&](const Str& part, std::vector<std::pair<std::vector<int>, SiteOp>>& out) {
    out.clear();
    std::vector<int> dags;
    for (const EOp& x : part) dags.push_back(x.dag);
    for (const auto& lab : labelings(int(part.size()))) {
      if (part.size() && !valid(part, lab)) continue;
      SiteOp s;
      if (!site_red(tr_, dags, lab, s)) continue;
      out.push_back({lab, s});
    }
  };
  auto split = [&](const Str& O, Str& A, Str& B, Str& C, Str& D) {
    for (const EOp& x : O) {
      const int w = side_of(x.orb);
      (w == 0 ? A : w == 1 ? B : w == 2 ? C : D).push_back(x);
    }
  };
  std::vector<std::pair<std::vector<int>, SiteOp>> vb, vc;
  // ---- rows of the right complementary operators: left normal x sites x C(O)
  std::vector<EOp> outR;
  for (int o = 0; o <= q; ++o) {
    outR.push_back({o, 1});
    outR.push_back({o, 0});
  }
  std::vector<std::pair<Str, std::vector<int>>> rkeys;
  rkeys.push_back({{}, {}});
  for (const EOp& o : outR) rkeys.push_back({{o}, {}});
  for (size_t a = 0; a < outR.size(); ++a)
    for (size_t b = a; b < outR.size(); ++b) {
      const Str pr{outR[a], outR[b]};
      for (const auto& lab : labelings(2))
        if (valid(pr, lab)) rkeys.push_back({pr, lab});
    }
  for (size_t a = 0; a < outR.size(); ++a)
    for (size_t b = a; b < outR.size(); ++b)
      for (size_t c = b; c < outR.size(); ++c) {
        const Str tr3{outR[a], outR[b], outR[c]};
        int nLops = 0;
        for (const EOp& x : tr3) nLops += x.orb < nL;
        if (nLops > 1) continue;
        for (const auto& lab : labelings(3))
          if (valid(tr3, lab)) rkeys.push_back({tr3, lab});
      }
  std::vector<EOp> elR;
  for (int o : rside.orbs) {
    elR.push_back({o, 1});
    elR.push_back({o, 0});
  }
  for (const auto& [O, lam] : rkeys) {
    const int n = int(O.size());
    const int kX = lab_rank(n, lam);
    int dN = 0;
    for (const EOp& x : O) dN += x.dag ? 1 : -1;
    std::vector<Part> parts;
    const std::string key = opkey('C', O, lam);
    if (n <= 2) {
      const int i = RL.find(key);
      if (i < 0) continue;
      parts.push_back({i, 1.0});
      if (n == 2 && kX == 0)  // the one-body string O (outside R) is counted elsewhere
        if (const Table16* F = strings_.find(O)) {
          const double c = tr_.coef(lnest(2, lam), F->v, 4);
          if (c != 0.0) parts.push_back({-1, -c});
        }
    } else {  // three outside factors: a sum of the block's elementary operators
      if (kX != 1) continue;
      for (const EOp& x : elR) {
        Str S = O;
        S.push_back(x);
        const Table16* F = strings_.find(S);
        if (!F) continue;
        const double c = tr_.coef(node(lnest(n, lam), "e", 0), F->v, 16);
        if (c != 0.0) parts.push_back({must(RL.find(opkey('N', Str{x}, {}))), c});
      }
      if (parts.empty()) continue;
    }
    Str A, B, C, D;
    split(O, A, B, C, D);
    const int nA = int(A.size());
    const int Did = final_op(fr, RL, n == 0 ? "H" : key, kX, -dN, n % 2, parts);
    const std::string src = node(lnest(n, lam), xleaf(kX), 0);
    site_variants(B, vb);
    site_variants(C, vc);
    for (const auto& alpha : labelings(nA)) {
      if (nA && !valid(A, alpha)) continue;
      const int kA = lab_rank(nA, alpha);
      int Aid = 0;
      if (nA == 1) {
        Aid = final_op(fl, LL, opkey('N', A, {}), 1, A[0].dag ? 1 : -1, 1, {{must(LL.find(opkey('N', A, {}))), 1.0}});
      } else if (nA == 2) {
        const int li = LL.find(opkey('P', A, alpha));
        if (li < 0) continue;
        const int dA = (A[0].dag ? 1 : -1) + (A[1].dag ? 1 : -1);
        Aid = final_op(fl, LL, opkey('P', A, alpha), kA, dA, 0, {{li, 1.0}});
      }
      for (const auto& [beta, Bs] : vb)
        for (const auto& [gamma, Cs] : vc)
          for (int k = 0; k <= 8; ++k) {
            if (!triangle(kA, Bs.k, k) || !triangle(Cs.k, kX, k)) continue;
            const std::string dst = node(node(lnest(nA, alpha), lnest(int(B.size()), beta), k),
                                         node(lnest(int(C.size()), gamma), xleaf(kX), k), 0);
            const double W = tr_.overlap(src, dst);
            if (std::abs(W) < 1e-14) continue;
            rows.push_back(Row{W, Aid, Did, k, Bs, Cs});
          }
    }
  }
  // ---- rows of the left complementary operators: C_L(O) x sites x right normal
  std::vector<EOp> sites, outL;
  for (int o : {p, q}) {
    sites.push_back({o, 1});
    sites.push_back({o, 0});
  }
  outL = sites;
  for (int o = q + 1; o < L_; ++o) {
    outL.push_back({o, 1});
    outL.push_back({o, 0});
  }
  std::vector<std::pair<Str, std::vector<int>>> lkeys;
  for (const EOp& o : outL) lkeys.push_back({{o}, {}});
  for (size_t a = 0; a < sites.size(); ++a)
    for (size_t b = a; b < outL.size(); ++b) {
      const Str pr{sites[a], outL[b]};
      for (const auto& lab : labelings(2))
        if (valid(pr, lab)) lkeys.push_back({pr, lab});
    }
  for (size_t a = 0; a < sites.size(); ++a)
    for (size_t b = a; b < sites.size(); ++b)
      for (size_t c = b; c < sites.size(); ++c) {
        const Str t3{sites[a], sites[b], sites[c]};
        for (const auto& lab : labelings(3))
          if (valid(t3, lab)) lkeys.push_back({t3, lab});
      }
  std::vector<EOp> elL;
  for (int o : lside.orbs) {
    elL.push_back({o, 1});
    elL.push_back({o, 0});
  }
  for (const auto& [O, lam] : lkeys) {
    const int n = int(O.size());
    const int kX = lab_rank(n, lam);
    int dN = 0;
    for (const EOp& x : O) dN += x.dag ? 1 : -1;
    std::vector<Part> parts;
    const std::string key = opkey('C', O, lam);
    if (n == 1) {
      const int i = LL.find(key);
      if (i < 0) continue;
      parts.push_back({i, 1.0});
      if (O[0].orb > q)  // the one-body strings (left factor, right factor) are counted on the right
        for (const EOp& x : elL) {
          Str S{x};
          S.push_back(O[0]);
          const Table16* F = strings_.find(S);
          if (!F) continue;
          const double c = tr_.coef(node("e", "e", 0), F->v, 4);
          if (c != 0.0) parts.push_back({must(LL.find(opkey('N', Str{x}, {}))), -c});
        }
    } else if (n == 2) {  // two left factors, no scalar part
      for (size_t a = 0; a < elL.size(); ++a)
        for (size_t b = a; b < elL.size(); ++b) {
          const Str pr{elL[a], elL[b]};
          Str S = pr;
          S.insert(S.end(), O.begin(), O.end());
          const Table16* F = strings_.find(S);
          if (!F) continue;
          for (const auto& mu : labelings(2)) {
            if (!valid(pr, mu) || mu[0] != kX) continue;
            const double c = tr_.coef(node(lnest(2, mu), lnest(2, lam), 0), F->v, 16);
            if (c != 0.0) parts.push_back({must(LL.find(opkey('P', pr, mu))), c});
          }
        }
      if (parts.empty()) continue;
    } else {  // three site factors, one left factor
      if (kX != 1) continue;
      for (const EOp& x : elL) {
        Str S{x};
        S.insert(S.end(), O.begin(), O.end());
        const Table16* F = strings_.find(S);
        if (!F) continue;
        const double c = tr_.coef(node("e", lnest(3, lam), 0), F->v, 16);
        if (c != 0.0) parts.push_back({must(LL.find(opkey('N', Str{x}, {}))), c});
      }
      if (parts.empty()) continue;
    }
    Str A, B, C, D;
    split(O, A, B, C, D);
    const int Aid = final_op(fl, LL, key, kX, -dN, n % 2, parts);
    int Did = 0, kD = 0;
    if (D.size() == 1) {
      Did = final_op(fr, RL, opkey('N', D, {}), 1, D[0].dag ? 1 : -1, 1, {{must(RL.find(opkey('N', D, {}))), 1.0}});
      kD = 1;
    }
    const std::string src = node(xleaf(kX), lnest(n, lam), 0);
    site_variants(B, vb);
    site_variants(C, vc);
    for (const auto& [beta, Bs] : vb)
      for (const auto& [gamma, Cs] : vc)
        for (int k = 0; k <= 8; ++k) {
          if (!triangle(kX, Bs.k, k) || !triangle(Cs.k, kD, k)) continue;
          const std::string dst = node(node(xleaf(kX), lnest(int(B.size()), beta), k),
                                       node(lnest(int(C.size()), gamma), lnest(int(D.size()), {}), k), 0);
          const double W = tr_.overlap(src, dst);
          if (std::abs(W) < 1e-14) continue;
          rows.push_back(Row{W, Aid, Did, k, Bs, Cs});
        }
  }
  if (iHL >= 0) rows.push_back(Row{1.0, fl.ids.at("H"), 0, 0, Isite, Isite});
  // ---- strings on the two sites only
  for (int nc1 = 0; nc1 <= 2; ++nc1)
    for (int na1 = 0; na1 <= 2; ++na1)
      for (int nc2 = 0; nc2 <= 2; ++nc2)
        for (int na2 = 0; na2 <= 2; ++na2) {
          const int n = nc1 + na1 + nc2 + na2;
          if (n != 2 && n != 4) continue;
          Str S, B, C;
          for (int i = 0; i < nc1; ++i) B.push_back({p, 1});
          for (int i = 0; i < na1; ++i) B.push_back({p, 0});
          for (int i = 0; i < nc2; ++i) C.push_back({q, 1});
          for (int i = 0; i < na2; ++i) C.push_back({q, 0});
          S = B;
          S.insert(S.end(), C.begin(), C.end());
          const Table16* F = strings_.find(S);
          if (!F) continue;
          site_variants(B, vb);
          site_variants(C, vc);
          for (const auto& [beta, Bs] : vb)
            for (const auto& [gamma, Cs] : vc)
              for (int k = 0; k <= 8; ++k) {
                if (!triangle(0, Bs.k, k) || !triangle(Cs.k, 0, k)) continue;
                const std::string t = node(node("0", lnest(int(B.size()), beta), k),
                                           node(lnest(int(C.size()), gamma), "0", k), 0);
                const double W = tr_.coef(t, F->v, 1 << n);
                if (std::abs(W) < 1e-14) continue;
                rows.push_back(Row{W, 0, 0, k, Bs, Cs});
              }
        }
  // ---- final arenas: one assembly step per side
  table.site_kind = SU2_SITE_ORBITAL;
  table.lops = fl.descs;
  table.rops = fr.descs;
  for (const Row& r : rows) {
    Term t;
    t.alpha = r.a;
    t.A = r.A;
    t.D = r.D;
    t.k = r.k;
    t.B = r.B;
    t.C = r.C;
    table.terms.push_back(t);
  }
  for (int side = 0; side < 2; ++side) {
    Final& f = side == 0 ? fl : fr;
    Side& sd = side == 0 ? lside : rside;
    RStep st;
    st.old_size = sd.arena ? sd.arena_size : sd.be->size();
    st.src_size = f.src_size;
    st.idents = f.idents;
    st.dst_size = f.lay.size;
    st.copies = f.groups;
    st.copy_terms = f.terms;
    double* kept = nullptr;
    std::string err = sd.arena ? sd.be->run_keep(st, sd.arena, &kept) : sd.be->run(st);
    if (!err.empty()) return err;
    SideOps& so = side == 0 ? Lops : Rops;
    so = SideOps();
    for (int oi = 1; oi < int(f.descs.size()); ++oi) {
      const OpDir& od = f.lay.ops[oi - 1];
      for (const auto& [bk, off] : od.blk) {
        const int qo = bk / 4096, qi = bk % 4096;
        so.index[SideOps::key(oi, qo, qi)] = int(so.blocks.size());
        so.blocks.push_back(OpBlock{oi, qo, qi, f.lay.sec[qo].dim, f.lay.sec[qi].dim, off});
      }
    }
    so.arena_size = f.lay.size;
    if (device_ >= 0) {
      so.host_values = false;
      so.dev_ready = sd.arena ? kept : sd.be->take_device();
    } else {
      so.host_values = true;
      so.arena = sd.be->take_host();
      so.arena.resize(size_t(so.arena_size));
    }
  }
  if (flops) *flops = lside.be->flops + rside.be->flops;
  return "";
}

}  // namespace

std::string build_abinitio(const su2_hamiltonian& H, const std::vector<std::vector<Sector>>& lchain,
                           const std::vector<std::vector<Sector>>& rchain, int device, void* stream,
                           int64_t t_budget_bytes, OpTable& table, SideOps& L, SideOps& R, double* renorm_flops) {
  if (!H.h || !H.eri) return "the ab initio model needs the integrals h and eri";
  if (H.n_left < 0 || H.n_right < 0) return "n_left and n_right must be >= 0";
  if (int(lchain.size()) != H.n_left + 1 || int(rchain.size()) != H.n_right + 1)
    return "the bond chains must have n_left + 1 and n_right + 1 bonds (vacuum first)";
  if (H.n_left + 2 + H.n_right > 1000) return "too many orbitals";
  try {
    Builder b(H, device, stream, t_budget_bytes);
    std::string err = b.grow(true, lchain, b.lside, H.mps_left);
    if (err.empty()) err = b.grow(false, rchain, b.rside, H.mps_right);
    if (err.empty()) err = b.assemble(table, L, R, renorm_flops);
    return err;
  } catch (const std::bad_alloc&) {
    return "host allocation failed";
  } catch (const std::exception& ex) {
    return ex.what();
  }
}

// ------------------------------------------------------------------ two-site sweep
// Blocks of every length kept on the device during a sweep: left block i
// holds orbitals 0 .. i-1, right block k the last k orbitals.
struct SweepBlocks {
  struct Rec {
    Layout lay;
    std::vector<int> orbs;
    double* arena = nullptr;
    int64_t size = 0;
  };
  std::unique_ptr<Builder> b;
  std::unique_ptr<RenormBackend> be;
  std::vector<Rec> Lb, Rb;
  // the MPS tensor that grew Lb[k] from Lb[k-1] (Rb[k] from Rb[k-1]): per
  // sector of the new bond, its stacked rows (previous sector, site state) x
  // dim, column-major; read by the wavefunction prediction
  std::vector<std::vector<std::vector<double>>> Lq, Rq;
  int L = 0, device = 0;
  ~SweepBlocks() {
    if (device >= 0) cudaSetDevice(device);
    for (auto& r : Lb) cudaFree(r.arena);
    for (auto& r : Rb) cudaFree(r.arena);
  }
};

namespace {

// left singular vectors and values of M (r x c, column-major), descending,
// by one-sided Jacobi rotations (Hestenes) on the narrower side
void svd_left(int r, int c, const std::vector<double>& M, std::vector<double>& U, std::vector<double>& sv) {
  const bool tr = c > r;               // rotate the columns of M^T: then U is the accumulated rotation
  const int rows = tr ? c : r, cols = tr ? r : c;
  std::vector<double> B(size_t(rows) * cols), V;
  for (int j = 0; j < cols; ++j)
    for (int i = 0; i < rows; ++i) B[size_t(i) + size_t(j) * rows] = tr ? M[size_t(j) + size_t(i) * r] : M[size_t(i) + size_t(j) * r];
  if (tr) {
    V.assign(size_t(cols) * cols, 0.0);
    for (int i = 0; i < cols; ++i) V[size_t(i) * (cols + 1)] = 1.0;
  }
  for (int sweep = 0; sweep < 80; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < cols; ++p)
      for (int q = p + 1; q < cols; ++q) {
        double a = 0, b = 0, g = 0;
        const double* bp = &B[size_t(p) * rows];
        const double* bq = &B[size_t(q) * rows];
        for (int i = 0; i < rows; ++i) {
          a += bp[i] * bp[i];
          b += bq[i] * bq[i];
          g += bp[i] * bq[i];
        }
        if (g == 0.0 || std::abs(g) <= 1e-15 * std::sqrt(a * b)) continue;
        off = std::max(off, std::abs(g) / std::sqrt(a * b));
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::abs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        double* xp = &B[size_t(p) * rows];
        double* xq = &B[size_t(q) * rows];
        for (int i = 0; i < rows; ++i) {
          const double u = xp[i], w = xq[i];
          xp[i] = cs * u - sn * w;
          xq[i] = sn * u + cs * w;
        }
        if (tr) {
          double* vp = &V[size_t(p) * cols];
          double* vq = &V[size_t(q) * cols];
          for (int i = 0; i < cols; ++i) {
            const double u = vp[i], w = vq[i];
            vp[i] = cs * u - sn * w;
            vq[i] = sn * u + cs * w;
          }
        }
      }
    if (off < 1e-15) break;
  }
  std::vector<double> nrm(static_cast<size_t>(cols));
  for (int j = 0; j < cols; ++j) {
    double x = 0;
    for (int i = 0; i < rows; ++i) x += B[size_t(i) + size_t(j) * rows] * B[size_t(i) + size_t(j) * rows];
    nrm[size_t(j)] = std::sqrt(x);
  }
  std::vector<int> ord(static_cast<size_t>(cols));
  for (int j = 0; j < cols; ++j) ord[size_t(j)] = j;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return nrm[size_t(a)] > nrm[size_t(b)]; });
  const int k = std::min(r, c);
  U.assign(size_t(r) * k, 0.0);
  sv.assign(size_t(k), 0.0);
  for (int x = 0; x < k; ++x) {
    const int j = ord[size_t(x)];
    sv[size_t(x)] = nrm[size_t(j)];
    for (int i = 0; i < r; ++i)
      U[size_t(i) + size_t(x) * r] = tr ? V[size_t(i) + size_t(j) * cols]
                                        : (nrm[size_t(j)] > 0 ? B[size_t(i) + size_t(j) * rows] / nrm[size_t(j)] : 0.0);
  }
}

}  // namespace

SweepBlocks* sweep_init(const su2_hamiltonian& H, const std::vector<std::vector<Sector>>& rchain, int device,
                        void* stream, int64_t budget, std::string& err) {
  const int L = H.n_left + 2 + H.n_right;
  if (int(rchain.size()) != L - 1) {
    err = "the initial right chain must hold the bonds of 0 .. L-2 orbitals";
    return nullptr;
  }
  auto* w = new SweepBlocks();
  w->L = L;
  w->device = device;
  try {
    w->b.reset(new Builder(H, device, stream, budget));
    w->be.reset(make_device_backend(device, stream, budget));
    w->Rb.resize(size_t(L - 1));
    w->Lb.resize(size_t(L - 1));
    w->Rq.resize(size_t(L - 1));
    w->Lq.resize(size_t(L - 1));
    w->Rb[0].lay.sec = rchain[0];
    w->Lb[0].lay.sec = std::vector<Sector>{Sector{0, 0, 1}};
    size_t pos = 0;
    for (int k = 1; k < L - 1; ++k) {
      SweepBlocks::Rec& o = w->Rb[size_t(k - 1)];
      Layout lay = o.lay;
      double* out = nullptr;
      std::vector<std::vector<double>> Q;
      if (H.mps_right) Q = w->b->step_tensors(rchain[size_t(k - 1)], rchain[size_t(k)], H.mps_right, &pos);
      else Q = w->b->seeded_tensors(false, k, rchain[size_t(k - 1)], rchain[size_t(k)]);
      if (Q.size() != rchain[size_t(k)].size()) {
        err = "bond dimension exceeds the states available from the previous bond";
        break;
      }
      err = w->b->step_block(false, k, L - k, rchain[size_t(k - 1)], rchain[size_t(k)], &Q, o.orbs, lay, *w->be,
                             o.arena, o.size, &out);
      if (!err.empty()) break;
      w->Rq[size_t(k)] = std::move(Q);
      SweepBlocks::Rec& r = w->Rb[size_t(k)];
      r.lay = lay;
      r.orbs = o.orbs;
      r.orbs.insert(r.orbs.begin(), L - k);
      r.arena = out;
      r.size = lay.size;
    }
  } catch (const std::exception& ex) {
    err = ex.what();
  }
  if (!err.empty()) {
    delete w;
    return nullptr;
  }
  return w;
}

void sweep_free(SweepBlocks* w) { delete w; }

std::string sweep_env(SweepBlocks* w, int i, OpTable& table, SideOps& Lops, SideOps& Rops, std::vector<Sector>& lsec,
                      std::vector<Sector>& rsec) {
  if (i < 0 || i > w->L - 2) return "window outside the chain";
  SweepBlocks::Rec& l = w->Lb[size_t(i)];
  SweepBlocks::Rec& r = w->Rb[size_t(w->L - 2 - i)];
  if (l.lay.sec.empty() || r.lay.sec.empty()) return "a block of the window has not been built";
  Builder& b = *w->b;
  b.lside.lay = l.lay;
  b.lside.orbs = l.orbs;
  b.lside.be = w->be.get();
  b.lside.arena = l.arena;
  b.lside.arena_size = l.size;
  b.rside.lay = r.lay;
  b.rside.orbs = r.orbs;
  b.rside.be = w->be.get();
  b.rside.arena = r.arena;
  b.rside.arena_size = r.size;
  try {
    std::string err = b.assemble(table, Lops, Rops, nullptr);
    if (!err.empty()) return err;
  } catch (const std::exception& ex) {
    return ex.what();
  }
  lsec = l.lay.sec;
  rsec = r.lay.sec;
  return "";
}

std::string sweep_split(const std::vector<Block>& blocks, const double* psi, const std::vector<Sector>& lsec,
                        const std::vector<Sector>& rsec, int N, int D, bool left, std::vector<Sector>& new_sec,
                        std::vector<std::vector<double>>& Q, double* discarded,
                        std::vector<std::vector<double>>* rest, int site_kind, int twoS) {
  std::vector<int> sN, sS;
  site_states(site_kind, sN, sS);
  const int ns = int(sN.size());
  struct Stk {
    int q, s, r0, d, j;  // sector, site state, first row, rows; j: coupled spin of the half
  };
  // the stacks (sector, site state) of one half with coupled spin j,
  // numbered on from tot
  auto stacks = [&](const std::vector<Sector>& sec, int Nq, int j, int& tot, std::vector<Stk>& v) {
    for (int qp = 0; qp < int(sec.size()); ++qp)
      for (int si = 0; si < ns; ++si)
        if (sec[qp].N + sN[si] == Nq && triangle(sec[qp].twoS, sS[si], j)) {
          v.push_back(Stk{qp, si, tot, sec[qp].dim, j});
          tot += sec[qp].dim;
        }
  };
  // the bond matrix of each sector (N_k, j) of the block that grows: moving
  // right, rows (a, s1) of the left half with j_L1 = j and columns (s2, b) of
  // every j_2R coupling with j to the target, j_2R ascending; moving left,
  // columns (s2, b) with j_2R = j and rows over every j_L1.  The coupled
  // states are orthonormal, so the singular values carry the multiplet weights.
  std::map<std::array<int, 6>, int> bidx;
  std::map<std::pair<int, int>, int> keys;
  for (int i = 0; i < int(blocks.size()); ++i) {
    const Block& B = blocks[i];
    bidx[{B.a, B.s1, B.s2, B.b, B.jL1, B.j2R}] = i;
    if (left) keys[{lsec[B.a].N + sN[B.s1], B.jL1}] = 1;
    else keys[{rsec[B.b].N + sN[B.s2], B.j2R}] = 1;
  }
  struct Sec {
    int Nk, j;
    std::vector<double> U, sv, M;  // M: the bond matrix (nr x nc, column-major)
    int rows, nr, nc;
  };
  std::vector<Sec> all;
  double total = 0.0;
  for (const auto& kv : keys) {
    const int Nk = kv.first.first, j = kv.first.second;
    int nown = 0, nother = 0;
    std::vector<Stk> own, other;
    stacks(left ? lsec : rsec, Nk, j, nown, own);
    for (int jo = std::abs(j - twoS); jo <= j + twoS; jo += 2) stacks(left ? rsec : lsec, N - Nk, jo, nother, other);
    const std::vector<Stk>& ls = left ? own : other;
    const std::vector<Stk>& rs = left ? other : own;
    const int nr = left ? nown : nother, nc = left ? nother : nown;
    std::vector<double> M(size_t(nr) * nc, 0.0);
    for (const Stk& x : ls)
      for (const Stk& y : rs) {
        auto it = bidx.find({x.q, x.s, y.s, y.q, x.j, y.j});
        if (it == bidx.end()) continue;
        const Block& B = blocks[it->second];
        for (int c = 0; c < B.cols; ++c)
          for (int r = 0; r < B.rows; ++r)
            M[size_t(x.r0 + r) + size_t(y.r0 + c) * nr] = psi[B.offset + r + int64_t(c) * B.rows];
      }
    Sec sc;
    sc.Nk = Nk;
    sc.j = j;
    sc.nr = nr;
    sc.nc = nc;
    if (left) {
      svd_left(nr, nc, M, sc.U, sc.sv);
      sc.rows = nr;
    } else {
      std::vector<double> Mt(M.size());
      for (int c = 0; c < nc; ++c)
        for (int r = 0; r < nr; ++r) Mt[size_t(c) + size_t(r) * nc] = M[size_t(r) + size_t(c) * nr];
      svd_left(nc, nr, Mt, sc.U, sc.sv);
      sc.rows = nc;
    }
    for (double x : sc.sv) total += x * x;
    if (rest) sc.M = std::move(M);
    all.push_back(std::move(sc));
  }
  // keep the D largest sigma^2; ties to the lower (N, 2S) sector, then the lower index
  struct Cand {
    double w;
    int N, j, sec, idx;
  };
  // singular values with sigma^2 <= 1e-24 of the total weight are never
  // kept: their singular vectors are arbitrary
  std::vector<Cand> cand;
  for (int q = 0; q < int(all.size()); ++q) {
    const int Nb = all[q].Nk;
    for (int x = 0; x < int(all[q].sv.size()); ++x) {
      const double w2 = all[q].sv[x] * all[q].sv[x];
      if (w2 > 1e-24 * total) cand.push_back(Cand{w2, Nb, all[q].j, q, x});
    }
  }
  std::stable_sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
    if (a.w != b.w) return a.w > b.w;
    if (a.N != b.N) return a.N < b.N;
    if (a.j != b.j) return a.j < b.j;
    return a.idx < b.idx;
  });
  std::map<int, int> nkeep;
  for (int x = 0; x < int(cand.size()) && x < D; ++x) nkeep[cand[x].sec] += 1;
  // discarded weight: the sum of the sigma^2 not kept (summed directly, so
  // that it is 0 when every non-zero singular value is kept)
  double dropped = 0.0;
  for (int q = 0; q < int(all.size()); ++q) {
    const auto it = nkeep.find(q);
    const int d = it == nkeep.end() ? 0 : it->second;
    for (int x = d; x < int(all[q].sv.size()); ++x) dropped += all[q].sv[x] * all[q].sv[x];
  }
  std::vector<std::pair<std::pair<int, int>, int>> order;  // ((N, 2S) of the new bond, sector)
  for (const auto& kv : nkeep) {
    const Sec& sc = all[size_t(kv.first)];
    order.push_back({{sc.Nk, sc.j}, kv.first});
  }
  std::sort(order.begin(), order.end());
  new_sec.clear();
  Q.clear();
  if (rest) rest->clear();
  for (const auto& o : order) {
    const Sec& sc = all[size_t(o.second)];
    const int d = nkeep[o.second];  // the d largest of this sector (descending order)
    new_sec.push_back(Sector{o.first.first, o.first.second, d});
    Q.emplace_back(sc.U.begin(), sc.U.begin() + size_t(sc.rows) * d);
    orthonormalize(Q.back(), sc.rows, d);  // removes the rounding of the rotations (the columns are already orthonormal to ~1e-15)
    if (!rest) continue;
    // the rest of the kept wavefunction: Q^T M (d x nc) moving right, M Q
    // (nr x d) moving left, column-major
    const std::vector<double>& q = Q.back();
    const int nr = sc.nr, nc = sc.nc;
    std::vector<double> C;
    if (left) {
      C.assign(size_t(d) * nc, 0.0);
      for (int c = 0; c < nc; ++c)
        for (int k = 0; k < d; ++k) {
          double acc = 0.0;
          for (int r = 0; r < nr; ++r) acc += q[size_t(r) + size_t(k) * nr] * sc.M[size_t(r) + size_t(c) * nr];
          C[size_t(k) + size_t(c) * d] = acc;
        }
    } else {
      C.assign(size_t(nr) * d, 0.0);
      for (int k = 0; k < d; ++k)
        for (int c = 0; c < nc; ++c) {
          const double qv = q[size_t(c) + size_t(k) * nc];
          if (qv == 0.0) continue;
          for (int r = 0; r < nr; ++r) C[size_t(r) + size_t(k) * nr] += sc.M[size_t(r) + size_t(c) * nr] * qv;
        }
    }
    rest->push_back(std::move(C));
  }
  if (discarded) *discarded = dropped;
  return new_sec.empty() ? "the wavefunction is zero" : "";
}

std::string sweep_grow(SweepBlocks* w, int i, bool left, const std::vector<Sector>& cur,
                       const std::vector<std::vector<double>>& Q) {
  const int L = w->L;
  SweepBlocks::Rec& o = left ? w->Lb[size_t(i)] : w->Rb[size_t(L - 2 - i)];
  SweepBlocks::Rec& n = left ? w->Lb[size_t(i + 1)] : w->Rb[size_t(L - 1 - i)];
  const int s = left ? i : i + 1;
  Layout lay = o.lay;
  double* out = nullptr;
  std::string err;
  try {
    err = w->b->step_block(left, 0, s, o.lay.sec, cur, &Q, o.orbs, lay, *w->be, o.arena, o.size, &out);
  } catch (const std::exception& ex) {
    err = ex.what();
  }
  if (!err.empty()) return err;
  cudaFree(n.arena);
  n.lay = lay;
  n.orbs = o.orbs;
  if (left) n.orbs.push_back(s);
  else n.orbs.insert(n.orbs.begin(), s);
  n.arena = out;
  n.size = lay.size;
  if (left) w->Lq[size_t(i + 1)] = Q;
  else w->Rq[size_t(L - 1 - i)] = Q;
  return "";
}

// Wavefunction prediction.  Moving right from window i the kept
// wavefunction is Q (Q^T M) per bond sector: Q became the grown left block,
// and C = Q^T M, with columns stacked (j_2R, right sector b, site s2), is
// expanded over the right block's MPS tensor, b = [s3 x r'] with rows
// stacked (r', s3), into the blocks (k, s2, s3, r', j', S_b) of window i+1.
// Moving left, C = M Q (rows (j_L1, left sector a, site s1)) is expanded over
// the left block's tensor, a = [a'' x s0], into the blocks
// (a'', s0, s1, k, S_a, j'') of window i-1.  The spins are recoupled,
// (j_k (s2 S_b)_j2R)_S -> ((j_k s2)_j' S_b)_S and ((S_a s1)_jL1 j_k)_S ->
// (S_a (s1 j_k)_j'')_S, by the 6j factor of `recouple`, which is exactly 1
// at S = 0 (one term, j' = S_b); no operator changes places, so no fermionic
// sign enters.  The guess is laid out in the next window's block order
// (build_blocks of its sectors).
std::string sweep_right_state(SweepBlocks* w, std::vector<std::vector<Sector>>& chain,
                              std::vector<std::vector<std::vector<double>>>& tensors) {
  chain.clear();
  tensors.clear();
  for (size_t k = 0; k < w->Rb.size(); ++k) {
    if (k > 0 && w->Rq[k].size() != w->Rb[k].lay.sec.size()) return "a right block's MPS tensor is not known";
    chain.push_back(w->Rb[k].lay.sec);
    tensors.push_back(k > 0 ? w->Rq[k] : std::vector<std::vector<double>>());
  }
  return "";
}

std::string sweep_predict(SweepBlocks* w, int i, bool right, const std::vector<Sector>& lsec,
                          const std::vector<Sector>& rsec, int N, const std::vector<Sector>& cur,
                          const std::vector<std::vector<double>>& rest, std::vector<double>& guess, int twoS) {
  const int L = w->L;
  const int nx = right ? i + 1 : i - 1;
  if (nx < 0 || nx > L - 2) return "no window to predict";
  return predict_guess(right, lsec, rsec, w->Lb[size_t(nx)].lay.sec, w->Rb[size_t(L - 2 - nx)].lay.sec,
                       right ? w->Rq[size_t(L - 2 - i)] : w->Lq[size_t(i)], N, SU2_SITE_ORBITAL, cur, rest, guess,
                       twoS);
}

namespace {
// <((j1 j2) j12, j3) J | (j1, (j2 j3) j23) J> (twos): the recoupling of three
// spins, (-1)^(j1+j2+j3+J) sqrt((2 j12+1)(2 j23+1)) {j1 j2 j12; j3 J j23}
double recouple(int j1, int j2, int j3, int J, int j12, int j23) {
  if (J == 0) return (j12 == j3 && j23 == j1) ? 1.0 : 0.0;
  const double sg = (((j1 + j2 + j3 + J) / 2) % 2) ? -1.0 : 1.0;
  return sg * std::sqrt(double(j12 + 1) * double(j23 + 1)) * sixj(j1, j2, j12, j3, J, j23);
}
}  // namespace

std::string predict_guess(bool right, const std::vector<Sector>& lsec, const std::vector<Sector>& rsec,
                          const std::vector<Sector>& nl, const std::vector<Sector>& nr,
                          const std::vector<std::vector<double>>& T, int N, int site_kind,
                          const std::vector<Sector>& cur, const std::vector<std::vector<double>>& rest,
                          std::vector<double>& guess, int twoS) {
  const std::vector<Sector>& tsec = right ? rsec : lsec;            // sectors the tensor produces
  const std::vector<Sector>& tprev = right ? nr : nl;                // its previous bond
  if (T.size() != tsec.size()) return "the MPS tensor of the adjacent block is not known";
  std::vector<Block> nb;
  int64_t nlen = 0;
  std::string err = build_blocks(nl, nr, site_kind, N, twoS, nb, nlen);
  if (!err.empty()) return err;
  std::map<std::array<int, 6>, int> bidx;
  for (int x = 0; x < int(nb.size()); ++x) bidx[{nb[x].a, nb[x].s1, nb[x].s2, nb[x].b, nb[x].jL1, nb[x].j2R}] = x;
  std::vector<int> sN, sS;
  site_states(site_kind, sN, sS);
  struct Stk {
    int q, s, r0, d, j;
  };
  auto stacks = [&](const std::vector<Sector>& sec, int Nq, int j, int& tot, std::vector<Stk>& v) {
    for (int qp = 0; qp < int(sec.size()); ++qp)
      for (int si = 0; si < int(sN.size()); ++si)
        if (sec[qp].N + sN[si] == Nq && triangle(sec[qp].twoS, sS[si], j)) {
          v.push_back(Stk{qp, si, tot, sec[qp].dim, j});
          tot += sec[qp].dim;
        }
  };
  guess.assign(size_t(nlen), 0.0);
  for (int qo = 0; qo < int(cur.size()); ++qo) {
    const int jk = cur[qo].twoS, d = cur[qo].dim;
    const int No = N - cur[qo].N;  // particles of the other half of window i
    // right: C's columns (b, s2) of window i's right half, j_2R ascending over
    // the spins that couple with j_k to S; left: C's rows (a, s1) likewise
    int tot = 0;
    std::vector<Stk> st;
    for (int jo = std::abs(jk - twoS); jo <= jk + twoS; jo += 2) stacks(right ? rsec : lsec, No, jo, tot, st);
    const std::vector<double>& C = rest[size_t(qo)];
    if (C.size() != size_t(tot) * d) return "prediction: the kept wavefunction does not match its stacks";
    for (const Stk& x : st) {
      const int S = tsec[size_t(x.q)].twoS, dq = tsec[size_t(x.q)].dim;
      const int ts = sS[size_t(x.s)];  // spin of the site between the kept half and the adjacent block
      int trows = 0;
      std::vector<Stk> tst;
      stacks(tprev, tsec[size_t(x.q)].N, S, trows, tst);
      const std::vector<double>& G = T[size_t(x.q)];
      if (G.size() != size_t(trows) * dq) return "prediction: an MPS tensor does not match its stacks";
      // the new coupled spin of the site with the kept half, and its weight:
      // right: (j_k (s2 S_b)_j2R)_S -> ((j_k s2)_j' S_b)_S; left: ((S_a s1)_jL1
      // j_k)_S -> (S_a (s1 j_k)_j'')_S
      std::vector<std::pair<int, double>> terms;
      for (int jn = std::abs(jk - ts); jn <= jk + ts; jn += 2) {
        if (!triangle(jn, S, twoS)) continue;
        const double wgt = right ? recouple(jk, ts, S, twoS, jn, x.j) : recouple(S, ts, jk, twoS, x.j, jn);
        if (wgt != 0.0) terms.push_back({jn, wgt});
      }
      for (const Stk& y : tst)
        for (const auto& tw : terms) {
          // right: block (qo, s2 = x.s, s3 = y.s, r' = y.q, j', S_b); left: (a'' = y.q, s0 = y.s, s1 = x.s, qo, S_a, j'')
          const auto it = right ? bidx.find({qo, x.s, y.s, y.q, tw.first, S})
                                : bidx.find({y.q, y.s, x.s, qo, S, tw.first});
          if (it == bidx.end()) return "prediction: a block of the next window is missing";
          const Block& B = nb[size_t(it->second)];
          double* out = guess.data() + B.offset;
          const double wgt = tw.second;
          if (right) {
            // out (d x dr') += wgt C[:, x.r0 : x.r0 + db] G[y.r0 : y.r0 + dr', :]^T
            for (int c = 0; c < B.cols; ++c)
              for (int m = 0; m < dq; ++m) {
                const double g = wgt * G[size_t(y.r0 + c) + size_t(m) * trows];
                if (g == 0.0) continue;
                const double* cc = &C[size_t(x.r0 + m) * d];
                for (int r = 0; r < B.rows; ++r) out[r + int64_t(c) * B.rows] += cc[r] * g;
              }
          } else {
            // out (da'' x d) += wgt G[y.r0 : y.r0 + da'', :] C[x.r0 : x.r0 + da, :]
            for (int c = 0; c < B.cols; ++c)
              for (int m = 0; m < dq; ++m) {
                const double cv = wgt * C[size_t(x.r0 + m) + size_t(c) * tot];
                if (cv == 0.0) continue;
                for (int r = 0; r < B.rows; ++r) out[r + int64_t(c) * B.rows] += G[size_t(y.r0 + r) + size_t(m) * trows] * cv;
              }
          }
        }
    }
  }
  return "";
}

}  // namespace su2
