// Host-side tables of the SU(2) two-site H.psi (arXiv:2309.16724):
// site operators (Sec. II.B), operator-table (Eq. 2), sector-table of psi
// (Sec. II.A), block operators (synthetic entries or renormalised from a
// seeded MPS, Sec. II.C), sector-task-table (Eq. 3) and sector-value table
// (Sec. II.C).  Integer decisions only select tasks; FP64 only fills values.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <tuple>

#include "su2_internal.h"

namespace su2 {

// ------------------------------------------------------------ generator
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
uint64_t splitmix(uint64_t x) { return mix64(x + kGamma); }
uint64_t block_key(uint64_t seed, uint64_t side, uint64_t op, uint64_t qo, uint64_t qi) {
  uint64_t h = splitmix(seed);
  h = splitmix(h ^ side);
  h = splitmix(h ^ op);
  return splitmix(h ^ ((qo << 32) | qi));
}
double uniform_elem(uint64_t key, uint64_t idx) {
  const uint64_t x = mix64(key + (idx + 1) * kGamma);
  return double(x >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// ------------------------------------------------------------ site operators
void site_states(int site_kind, std::vector<int>& N, std::vector<int>& twoS) {
  if (site_kind == SU2_SITE_SPIN_HALF) {
    N = {1};
    twoS = {1};
  } else {
    N = {0, 1, 2};
    twoS = {0, 1, 0};
  }
}

// Adjoint tensor T^dag_q = (-1)^{k-q} (T_{-q})^+ in the CG form of
// Wigner-Eckart: <a||T^dag||b> = (-1)^{(S_b+k-S_a)/2} sqrt((S_b+1)/(S_a+1)) <b||T||a>.
static void adjoint_red(const double in[3][3], int n, int k, const std::vector<int>& tw, double out[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) out[a][b] = 0.0;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      if (in[b][a] == 0.0) continue;
      const int e = tw[b] + k - tw[a];
      const double sg = ((e / 2) % 2) ? -1.0 : 1.0;
      out[a][b] = sg * std::sqrt(double(tw[b] + 1) / double(tw[a] + 1)) * in[b][a];
    }
}

SiteOp site_adjoint(const SiteOp& op, int site_kind) {
  std::vector<int> N, tw;
  site_states(site_kind, N, tw);
  SiteOp r = op;
  r.dN = -op.dN;
  adjoint_red(op.red, op.n, op.k, tw, r.red);
  return r;
}

SiteOp site_op(int site_kind, const char* name) {
  SiteOp o;
  std::string s(name);
  if (site_kind == SU2_SITE_SPIN_HALF) {
    o.n = 1;
    if (s == "I") o.red[0][0] = 1.0;
    else if (s == "S") { o.k = 2; o.red[0][0] = std::sqrt(0.75); }
    else if (s == "n") o.red[0][0] = 1.0;
    else if (s == "S2") o.red[0][0] = 0.75;
    return o;
  }
  o.n = 3;
  if (s == "I") { o.red[0][0] = o.red[1][1] = o.red[2][2] = 1.0; }
  else if (s == "n") { o.red[1][1] = 1.0; o.red[2][2] = 2.0; }
  else if (s == "dbl") { o.red[2][2] = 1.0; }
  else if (s == "cdag") { o.k = 1; o.dN = 1; o.parity = 1; o.red[1][0] = 1.0; o.red[2][1] = -std::sqrt(2.0); }
  else if (s == "c") { o = site_adjoint(site_op(site_kind, "cdag"), site_kind); }
  else if (s == "S") { o.k = 2; o.red[1][1] = std::sqrt(0.75); }
  else if (s == "S2") { o.red[1][1] = 0.75; }
  else if (s == "pair") { o.dN = 2; o.red[2][0] = std::sqrt(2.0); }
  else if (s == "pairdag") { o = site_adjoint(site_op(site_kind, "pair"), site_kind); }
  return o;
}

// ------------------------------------------------------------ operator tables
namespace {

struct TableBuilder {
  OpTable t;
  int add(bool left, const BlockOp& op) {
    auto& v = left ? t.lops : t.rops;
    v.push_back(op);
    return int(v.size()) - 1;
  }
  int add_random_pair(bool left, const std::string& name, int k, int dN, int parity) {
    BlockOp a{name, k, dN, parity, OP_RANDOM, -1};
    const int i = add(left, a);
    BlockOp b{name + "^+", k, -dN, parity, OP_ADJOINT, i};
    add(left, b);
    return i;
  }
  int adjoint_id(bool left, int id) const {
    const auto& v = left ? t.lops : t.rops;
    const BlockOp& op = v[id];
    if (op.kind == OP_IDENTITY || op.kind == OP_HAM) return id;
    if (op.kind == OP_ADJOINT) return op.base;
    for (size_t j = 0; j < v.size(); ++j)
      if (v[j].kind == OP_ADJOINT && v[j].base == id) return int(j);
    return -1;
  }
  void term(double alpha, int A, const SiteOp& B, const SiteOp& C, int D, int k) {
    Term x;
    x.alpha = alpha; x.A = A; x.B = B; x.C = C; x.D = D; x.k = k;
    t.terms.push_back(x);
  }
  // term and its Hermitian conjugate: sign (-1)^{pX pY + pA pB + pC pD}
  void term_hc(double alpha, int A, const SiteOp& B, const SiteOp& C, int D, int k) {
    term(alpha, A, B, C, D, k);
    const int pA = t.lops[A].parity, pD = t.rops[D].parity, pB = B.parity, pC = C.parity;
    const int e = (pA + pB) * (pC + pD) + pA * pB + pC * pD;
    term(e % 2 ? -alpha : alpha, adjoint_id(true, A), site_adjoint(B, t.site_kind), site_adjoint(C, t.site_kind),
         adjoint_id(false, D), k);
  }
};

std::string str(const char* a, int i) { return std::string(a) + std::to_string(i); }

}  // namespace

OpTable make_table(const su2_hamiltonian& H, int site_kind) {
  TableBuilder b;
  b.t.site_kind = site_kind;
  auto so = [&](const char* n) { return site_op(site_kind, n); };
  if (H.model == SU2_MODEL_HEISENBERG) {
    for (int side = 0; side < 2; ++side) {
      b.add(side == 0, BlockOp{"I", 0, 0, 0, OP_IDENTITY, -1});
      b.add(side == 0, BlockOp{"H", 0, 0, 0, OP_MPS_RENORM, -1});
      b.add(side == 0, BlockOp{"S", 2, 0, 0, OP_MPS_RENORM, -1});
    }
    const double c = -std::sqrt(3.0) * H.J;  // S_a.S_b = -sqrt(3) [S_a x S_b]^0
    b.term(1.0, 1, so("I"), so("I"), 0, 0);  // H_L
    b.term(c, 2, so("S"), so("I"), 0, 0);    // S_L.s1
    b.term(c, 0, so("S"), so("S"), 0, 2);    // s1.s2
    b.term(c, 0, so("I"), so("S"), 2, 0);    // s2.S_R
    b.term(1.0, 0, so("I"), so("I"), 1, 0);  // H_R
    return b.t;
  }
  if (H.model == SU2_MODEL_CASIMIR_S2 || H.model == SU2_MODEL_CASIMIR_N) {
    for (int side = 0; side < 2; ++side) {
      b.add(side == 0, BlockOp{"I", 0, 0, 0, OP_IDENTITY, -1});
      b.add(side == 0, BlockOp{"S", 2, 0, 0, OP_SPINTOT, -1});
      b.add(side == 0, BlockOp{"N", 0, 0, 0, OP_NUMTOT, -1});
    }
    if (H.model == SU2_MODEL_CASIMIR_N) {
      const SiteOp n = so("n");
      b.term(1.0, 2, so("I"), so("I"), 0, 0);
      b.term(1.0, 0, n, so("I"), 0, 0);
      b.term(1.0, 0, so("I"), n, 0, 0);
      b.term(1.0, 0, so("I"), so("I"), 2, 0);
      return b.t;
    }
    b.add(true, BlockOp{"S2", 0, 0, 0, OP_SPINTOT, -1});
    b.add(false, BlockOp{"S2", 0, 0, 0, OP_SPINTOT, -1});
    const double c = -std::sqrt(3.0);
    const SiteOp S = so("S"), S2 = so("S2"), I = so("I");
    b.term(1.0, 3, I, I, 0, 0);
    b.term(1.0, 0, S2, I, 0, 0);
    b.term(1.0, 0, I, S2, 0, 0);
    b.term(1.0, 0, I, I, 3, 0);
    b.term(2 * c, 1, S, I, 0, 0);
    b.term(2 * c, 1, I, S, 0, 2);
    b.term(2 * c, 1, I, I, 1, 2);
    b.term(2 * c, 0, S, S, 0, 2);
    b.term(2 * c, 0, S, I, 1, 2);
    b.term(2 * c, 0, I, S, 1, 0);
    return b.t;
  }
  // ab initio skeleton: normal operators on the left block, complementary on
  // the right; families F1..F9 in the canonical order shared with the tests
  const int nL = H.n_left, nR = H.n_right;
  const SiteOp I = so("I"), n = so("n"), dbl = so("dbl"), cd = so("cdag"), c = so("c"), S = so("S"),
               pair = so("pair"), pairdag = so("pairdag");
  const int IL = b.add(true, BlockOp{"I", 0, 0, 0, OP_IDENTITY, -1});
  const int HL = b.add(true, BlockOp{"H", 0, 0, 0, OP_HAM, -1});
  const int IR = b.add(false, BlockOp{"I", 0, 0, 0, OP_IDENTITY, -1});
  const int HR = b.add(false, BlockOp{"H", 0, 0, 0, OP_HAM, -1});
  const double wL1 = 1.0 / std::sqrt(double(nL)), wL2 = 1.0 / double(nL), wR1 = 1.0 / std::sqrt(double(nR));
  b.term(1.0, HL, I, I, IR, 0);  // F1
  b.term(1.0, IL, I, I, HR, 0);
  b.term(0.5, IL, n, I, IR, 0);  // F2
  b.term(0.5, IL, dbl, I, IR, 0);
  b.term(0.5, IL, I, n, IR, 0);
  b.term(0.5, IL, I, dbl, IR, 0);
  b.term_hc(0.5, IL, cd, c, IR, 1);  // F3
  b.term(0.5, IL, S, S, IR, 2);
  b.term(0.5, IL, n, n, IR, 0);
  b.term_hc(0.5, IL, pair, pairdag, IR, 0);
  std::vector<int> aplus(nL);
  for (int i = 0; i < nL; ++i) {  // F4
    aplus[i] = b.add_random_pair(true, str("a+_", i), 1, +1, 1);
    const int sb = b.add_random_pair(false, str("Sbar_", i), 1, -1, 1);
    b.term_hc(wL1, aplus[i], I, I, sb, 1);
  }
  for (int i = 0; i < nL; ++i) {  // F5
    for (int k = 0; k <= 2; k += 2) {
      const int q = b.add_random_pair(false, str("Qp_", i), k, 0, 0);
      b.term_hc(wL1, aplus[i], c, I, q, k);
    }
    for (int k = 0; k <= 2; k += 2) {
      const int q = b.add_random_pair(false, str("Qq_", i), k, 0, 0);
      b.term_hc(wL1, aplus[i], I, c, q, 1);
    }
  }
  for (int i = 0; i < nL; ++i)  // F6
    for (int j = i; j < nL; ++j) {
      for (int k = 0; k <= 2; k += 2) {
        if (k == 2 && i == j) continue;
        const int A = b.add_random_pair(true, "A", k, +2, 0);
        const int P = b.add_random_pair(false, "P", k, -2, 0);
        b.term_hc(wL2, A, I, I, P, k);
      }
      for (int k = 0; k <= 2; k += 2) {
        const int B = b.add_random_pair(true, "B", k, 0, 0);
        const int Q = b.add_random_pair(false, "Q", k, 0, 0);
        b.term_hc(wL2, B, I, I, Q, k);
      }
    }
  for (int l = 0; l < nR; ++l) {  // F7
    const int SL = b.add_random_pair(true, str("S_", l), 1, +1, 1);
    const int aR = b.add_random_pair(false, str("a~_", l), 1, -1, 1);
    b.term_hc(wR1, SL, I, I, aR, 1);
  }
  const int sp = b.add_random_pair(false, "Sbar_p", 1, -1, 1);  // F8
  b.term_hc(0.5, IL, cd, I, sp, 1);
  const int sq = b.add_random_pair(false, "Sbar_q", 1, -1, 1);
  b.term_hc(0.5, IL, I, cd, sq, 0);
  const int Sp = b.add_random_pair(true, "S_p", 1, +1, 1);  // F9
  b.term_hc(0.5, Sp, c, I, IR, 0);
  const int Sq = b.add_random_pair(true, "S_q", 1, +1, 1);
  b.term_hc(0.5, Sq, I, c, IR, 1);
  return b.t;
}

// ------------------------------------------------------------ psi blocks
std::string build_blocks(const std::vector<Sector>& left, const std::vector<Sector>& right, int site_kind, int N,
                         int twoS, std::vector<Block>& blocks, int64_t& psi_len) {
  std::vector<int> sN, sS;
  site_states(site_kind, sN, sS);
  blocks.clear();
  int64_t off = 0;
  const int ns = int(sN.size());
  for (int a = 0; a < int(left.size()); ++a)
    for (int s1 = 0; s1 < ns; ++s1)
      for (int s2 = 0; s2 < ns; ++s2)
        for (int b = 0; b < int(right.size()); ++b) {
          if (left[a].N + sN[s1] + sN[s2] + right[b].N != N) continue;
          for (int jL1 = std::abs(left[a].twoS - sS[s1]); jL1 <= left[a].twoS + sS[s1]; jL1 += 2)
            for (int j2R = std::abs(sS[s2] - right[b].twoS); j2R <= sS[s2] + right[b].twoS; j2R += 2) {
              if (!triangle(jL1, j2R, twoS)) continue;
              blocks.push_back(Block{a, s1, s2, b, jL1, j2R, left[a].dim, right[b].dim, off});
              off += int64_t(left[a].dim) * right[b].dim;
            }
        }
  psi_len = off;
  return "";
}

// ------------------------------------------------------------ block operators
namespace {

void add_block(SideOps& so, int op, int qo, int qi, int rows, int cols) {
  OpBlock blk{op, qo, qi, rows, cols, so.arena_size};
  so.index[SideOps::key(op, qo, qi)] = int(so.blocks.size());
  so.blocks.push_back(blk);
  int64_t n = int64_t(rows) * cols;
  n = (n + 1) & ~int64_t(1);  // keep every block 16-byte aligned
  so.arena_size += n;
  if (so.host_values) so.arena.resize(size_t(so.arena_size), 0.0);
}

// structurally allowed (out, in) sector pairs of an operator
std::vector<std::pair<int, int>> allowed(const BlockOp& op, const std::vector<Sector>& sec) {
  std::vector<std::pair<int, int>> r;
  for (int qi = 0; qi < int(sec.size()); ++qi)
    for (int qo = 0; qo < int(sec.size()); ++qo)
      if (sec[qo].N == sec[qi].N + op.dN && triangle(sec[qi].twoS, op.k, sec[qo].twoS)) r.emplace_back(qo, qi);
  return r;
}

}  // namespace

// Q factor (positive diagonal of R) of a rows x cols column-major matrix by
// classical Gram-Schmidt applied twice.
void orthonormalize(std::vector<double>& G, int rows, int cols) {
  for (int c = 0; c < cols; ++c) {
    double* gc = &G[size_t(c) * rows];
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<double> h(c, 0.0);
      for (int p = 0; p < c; ++p) {
        const double* gp = &G[size_t(p) * rows];
        double s = 0.0;
        for (int r = 0; r < rows; ++r) s += gp[r] * gc[r];
        h[p] = s;
      }
      for (int p = 0; p < c; ++p) {
        const double* gp = &G[size_t(p) * rows];
        for (int r = 0; r < rows; ++r) gc[r] -= h[p] * gp[r];
      }
    }
    double nrm = 0.0;
    for (int r = 0; r < rows; ++r) nrm += gc[r] * gc[r];
    nrm = std::sqrt(nrm);
    for (int r = 0; r < rows; ++r) gc[r] /= nrm;
  }
}

std::vector<double> seeded_mps_tensor(uint64_t seed, uint64_t side, int step, int qo, int r0, int d) {
  std::vector<double> G(size_t(r0) * d);
  const uint64_t key = block_key(seed, side, uint64_t(step), uint64_t(qo), 0);
  for (int c = 0; c < d; ++c)
    for (int r = 0; r < r0; ++r) G[size_t(r) + size_t(c) * r0] = uniform_elem(key, uint64_t(r) + uint64_t(c) * r0);
  orthonormalize(G, r0, d);
  return G;
}

namespace {

struct Mat {
  int r = 0, c = 0;
  std::vector<double> a;  // column-major
  Mat() = default;
  Mat(int rr, int cc) : r(rr), c(cc), a(size_t(rr) * cc, 0.0) {}
  double& operator()(int i, int j) { return a[size_t(j) * r + i]; }
  double operator()(int i, int j) const { return a[size_t(j) * r + i]; }
};

// C = A^T B (A: n x p, B: n x q)
Mat atb(const Mat& A, const Mat& B) {
  Mat C(A.c, B.c);
  for (int j = 0; j < B.c; ++j)
    for (int i = 0; i < A.c; ++i) {
      double s = 0.0;
      for (int k = 0; k < A.r; ++k) s += A(k, i) * B(k, j);
      C(i, j) = s;
    }
  return C;
}
Mat ab(const Mat& A, const Mat& B) {
  Mat C(A.r, B.c);
  for (int j = 0; j < B.c; ++j)
    for (int k = 0; k < A.c; ++k) {
      const double b = B(k, j);
      if (b == 0.0) continue;
      for (int i = 0; i < A.r; ++i) C(i, j) += A(i, k) * b;
    }
  return C;
}

struct Stack {  // one (previous sector, site state) slot of a stacked MPS tensor row range
  int qp, s, r0, d;
};

// One growth step of a Heisenberg block: its {H, S} on bond `prev` (have =
// false for the empty block) projected by the MPS tensor Q (per new sector,
// the stacked rows (previous sector, site state) x dim) onto bond `cur`.
// left: block x site with the W9j^(l) factor; right: site x block, W9j^(r).
void heis_step(const std::vector<Sector>& prev, const std::vector<Sector>& cur, const std::vector<Mat>& Q, bool left,
               double J, bool have, std::map<std::pair<int, int>, Mat>& Hc, std::map<std::pair<int, int>, Mat>& Sc) {
  const int kind = SU2_SITE_SPIN_HALF;
  std::vector<int> sN, sS;
  site_states(kind, sN, sS);
  const SiteOp I = site_op(kind, "I"), Sop = site_op(kind, "S");
  std::vector<std::vector<Stack>> rows(cur.size());
  for (int qo = 0; qo < int(cur.size()); ++qo) {
    int r0 = 0;
    for (int qp = 0; qp < int(prev.size()); ++qp)
      for (int s = 0; s < int(sN.size()); ++s)
        if (prev[qp].N + sN[s] == cur[qo].N && triangle(prev[qp].twoS, sS[s], cur[qo].twoS)) {
          rows[qo].push_back(Stack{qp, s, r0, prev[qp].dim});
          r0 += prev[qp].dim;
        }
  }
  // coupled-basis reduced matrix of [O x s]^K (left) / [s x O]^K (right)
  auto coupled = [&](int qo, int qi, const std::map<std::pair<int, int>, Mat>* O, int kO, const SiteOp& so, int K) {
    Mat M(Q[qo].r, Q[qi].r);
    const int Sout = cur[qo].twoS, Sin = cur[qi].twoS;
    for (const Stack& ro : rows[qo])
      for (const Stack& ri : rows[qi]) {
        const double sv = so.red[ro.s][ri.s];
        if (sv == 0.0) continue;
        const Mat* Ob = nullptr;
        if (O) {
          auto it = O->find({ro.qp, ri.qp});
          if (it == O->end()) continue;
          Ob = &it->second;
        } else if (ro.qp != ri.qp) {
          continue;
        }
        const int Sli = prev[ri.qp].twoS, Slo = prev[ro.qp].twoS;
        const double cf = left ? ctilde(Sli, sS[ri.s], Sin, kO, so.k, K, Slo, sS[ro.s], Sout)
                               : ctilde(sS[ri.s], Sli, Sin, so.k, kO, K, sS[ro.s], Slo, Sout);
        if (cf == 0.0) continue;
        const double f = cf * sv;
        for (int c = 0; c < ri.d; ++c)
          for (int r = 0; r < ro.d; ++r) M(ro.r0 + r, ri.r0 + c) += f * (Ob ? (*Ob)(r, c) : (r == c ? 1.0 : 0.0));
      }
    return M;
  };
  std::map<std::pair<int, int>, Mat> Hn, Sn;
  for (int qo = 0; qo < int(cur.size()); ++qo)
    for (int qi = 0; qi < int(cur.size()); ++qi) {
      if (cur[qo].N != cur[qi].N) continue;
      if (cur[qo].twoS == cur[qi].twoS) {
        Mat M(Q[qo].r, Q[qi].r);
        if (have) {
          Mat X = coupled(qo, qi, &Hc, 0, I, 0);
          for (size_t i = 0; i < M.a.size(); ++i) M.a[i] += X.a[i];
          X = coupled(qo, qi, &Sc, 2, Sop, 0);
          const double c = -std::sqrt(3.0) * J;
          for (size_t i = 0; i < M.a.size(); ++i) M.a[i] += c * X.a[i];
        }
        Hn[{qo, qi}] = ab(atb(Q[qo], M), Q[qi]);
      }
      if (triangle(cur[qi].twoS, 2, cur[qo].twoS)) {
        Mat X = coupled(qo, qi, nullptr, 0, Sop, 2);
        Sn[{qo, qi}] = ab(atb(Q[qo], X), Q[qi]);
      }
    }
  Hc.swap(Hn);
  Sc.swap(Sn);
}

// the stacked rows (previous sector, site state) of every sector of `cur`
std::vector<int> stacked_rows(const std::vector<Sector>& prev, const std::vector<Sector>& cur, int kind) {
  std::vector<int> sN, sS;
  site_states(kind, sN, sS);
  std::vector<int> r(cur.size(), 0);
  for (size_t qo = 0; qo < cur.size(); ++qo)
    for (const Sector& p : prev)
      for (size_t s = 0; s < sN.size(); ++s)
        if (p.N + sN[s] == cur[qo].N && triangle(p.twoS, sS[s], cur[qo].twoS)) r[qo] += p.dim;
  return r;
}

// Renormalised Heisenberg block operators {H, S} grown over the bond chain
// by the seeded MPS tensors.
std::string heisenberg_ops(const std::vector<std::vector<Sector>>& chain, bool left, const su2_hamiltonian& H,
                           std::map<std::pair<int, int>, Mat>& Hout, std::map<std::pair<int, int>, Mat>& Sout) {
  std::map<std::pair<int, int>, Mat> Hc, Sc;
  for (size_t k = 1; k < chain.size(); ++k) {
    const auto& cur = chain[k];
    const std::vector<int> r0 = stacked_rows(chain[k - 1], cur, SU2_SITE_SPIN_HALF);
    std::vector<Mat> Q(cur.size());
    for (int qo = 0; qo < int(cur.size()); ++qo) {
      const int d = cur[qo].dim;
      if (r0[qo] < d) return "bond dimension exceeds the states available from the previous bond";
      Q[qo] = Mat(r0[qo], d);
      Q[qo].a = seeded_mps_tensor(H.seed, left ? 2 : 3, int(k), qo, r0[qo], d);
    }
    heis_step(chain[k - 1], cur, Q, left, H.J, k > 1, Hc, Sc);
  }
  Hout.swap(Hc);
  Sout.swap(Sc);
  return "";
}

}  // namespace

std::string build_side_ops(const OpTable& t, bool left_side, const std::vector<std::vector<Sector>>& chain,
                           const su2_hamiltonian& H, SideOps& out, bool host_values) {
  const auto& ops = left_side ? t.lops : t.rops;
  const std::vector<Sector>& sec = chain.back();
  const uint64_t side = left_side ? 0 : 1;
  out = SideOps();
  for (const auto& op : ops)
    if (op.kind == OP_MPS_RENORM || op.kind == OP_SPINTOT || op.kind == OP_NUMTOT) host_values = true;
  out.host_values = host_values;
  std::map<std::pair<int, int>, Mat> hH, hS;
  bool heis = false;
  for (const auto& op : ops) heis |= (op.kind == OP_MPS_RENORM);
  if (heis) {
    std::string err = heisenberg_ops(chain, left_side, H, hH, hS);
    if (!err.empty()) return err;
  }
  for (int oid = 0; oid < int(ops.size()); ++oid) {
    const BlockOp& op = ops[oid];
    if (op.kind == OP_IDENTITY) continue;
    if (op.kind == OP_RANDOM) {
      for (auto [qo, qi] : allowed(op, sec)) {
        const int ro = sec[qo].dim, ci = sec[qi].dim;
        add_block(out, oid, qo, qi, ro, ci);
        const double s = 1.0 / std::sqrt(double(std::max(ro, ci)));
        const uint64_t key = block_key(H.seed, side, uint64_t(oid), uint64_t(qo), uint64_t(qi));
        if (!host_values) {
          out.gen.push_back(GenBlock{out.blocks.back().off, ro, ci, 0, 0, key, s, 0.0});
          continue;
        }
        double* m = &out.arena[out.blocks.back().off];
        for (int64_t i = 0; i < int64_t(ro) * ci; ++i) m[i] = uniform_elem(key, uint64_t(i)) * s;
      }
    } else if (op.kind == OP_HAM) {
      for (int q = 0; q < int(sec.size()); ++q) {
        const int d = sec[q].dim;
        add_block(out, oid, q, q, d, d);
        const double s = 1.0 / std::sqrt(double(d));
        const uint64_t key = block_key(H.seed, side, uint64_t(oid), uint64_t(q), uint64_t(q));
        if (!host_values) {
          out.gen.push_back(GenBlock{out.blocks.back().off, d, d, 1, 0, key, s, 0.0});
          continue;
        }
        double* m = &out.arena[out.blocks.back().off];
        std::vector<double> X(size_t(d) * d);
        for (int64_t i = 0; i < int64_t(d) * d; ++i) X[i] = uniform_elem(key, uint64_t(i)) * s;
        for (int c = 0; c < d; ++c)
          for (int r = 0; r < d; ++r) m[r + size_t(c) * d] = 0.1 * (X[r + size_t(c) * d] + X[c + size_t(r) * d]);
        for (int r = 0; r < d; ++r) m[r + size_t(r) * d] += (2.0 * r) / d;
      }
    } else if (op.kind == OP_MPS_RENORM) {
      const auto& src = (op.name == "H") ? hH : hS;
      for (auto [qo, qi] : allowed(op, sec)) {
        add_block(out, oid, qo, qi, sec[qo].dim, sec[qi].dim);
        auto it = src.find({qo, qi});
        if (it != src.end()) std::copy(it->second.a.begin(), it->second.a.end(), &out.arena[out.blocks.back().off]);
      }
    } else if (op.kind == OP_SPINTOT || op.kind == OP_NUMTOT) {
      for (auto [qo, qi] : allowed(op, sec)) {
        add_block(out, oid, qo, qi, sec[qo].dim, sec[qi].dim);
        if (qo != qi) continue;
        double val;
        const double j = sec[qi].twoS / 2.0;
        if (op.kind == OP_NUMTOT) val = double(sec[qi].N);
        else if (op.name == "S2") val = j * (j + 1);
        else val = std::sqrt(j * (j + 1));
        double* m = &out.arena[out.blocks.back().off];
        for (int r = 0; r < sec[qi].dim; ++r) m[r + size_t(r) * sec[qi].dim] = val;
      }
    }
  }
  // adjoint tensors, from their base operators
  std::unordered_map<int64_t, size_t> gen_at;  // arena offset -> generated block
  for (size_t g = 0; g < out.gen.size(); ++g) gen_at[out.gen[g].off] = g;
  for (int oid = 0; oid < int(ops.size()); ++oid) {
    const BlockOp& op = ops[oid];
    if (op.kind != OP_ADJOINT) continue;
    const int k = ops[op.base].k;
    for (auto [qo, qi] : allowed(ops[op.base], sec)) {
      // base block (qo <- qi) gives adjoint block (qi <- qo)
      const int src = out.find(op.base, qo, qi);
      const int Sa = sec[qi].twoS, Sb = sec[qo].twoS;
      const int e = Sb + k - Sa;
      const double f = (((e / 2) % 2) ? -1.0 : 1.0) * std::sqrt(double(Sb + 1) / double(Sa + 1));
      const int ro = sec[qi].dim, co = sec[qo].dim;
      add_block(out, oid, qi, qo, ro, co);
      if (!host_values) {
        // generated from the base block's own entries (no arena read), so
        // that any range of blocks can be generated on its own
        const GenBlock& b = out.gen[gen_at.at(out.blocks[src].off)];
        if (b.kind == 2) return "an adjoint of an adjoint operator";
        out.gen.push_back(GenBlock{out.blocks.back().off, ro, co, 2, b.kind, b.key, f, b.scale});
        continue;
      }
      double* m = &out.arena[out.blocks.back().off];
      const double* s = &out.arena[out.blocks[src].off];  // co x ro  (rows qo, cols qi)
      for (int c = 0; c < co; ++c)
        for (int r = 0; r < ro; ++r) m[r + size_t(c) * ro] = f * s[c + size_t(r) * co];
    }
  }
  return "";
}

std::string heis_grow(const HeisBlock& old, const std::vector<Sector>& cur, const std::vector<std::vector<double>>& Q,
                      bool left, double J, HeisBlock& out) {
  const std::vector<int> r0 = stacked_rows(old.sec, cur, SU2_SITE_SPIN_HALF);
  if (Q.size() != cur.size()) return "MPS tensor does not match the new bond";
  std::vector<Mat> Qm(cur.size());
  for (size_t qo = 0; qo < cur.size(); ++qo) {
    if (r0[qo] < cur[qo].dim) return "bond dimension exceeds the states available from the previous bond";
    if (Q[qo].size() != size_t(r0[qo]) * cur[qo].dim) return "MPS tensor does not match the stacked rows of its sector";
    Qm[qo] = Mat(r0[qo], cur[qo].dim);
    Qm[qo].a = Q[qo];
  }
  std::map<std::pair<int, int>, Mat> Hc, Sc;
  for (const auto& kv : old.H) {
    Mat m(old.sec[kv.first.first].dim, old.sec[kv.first.second].dim);
    m.a = kv.second;
    Hc[kv.first] = std::move(m);
  }
  for (const auto& kv : old.S) {
    Mat m(old.sec[kv.first.first].dim, old.sec[kv.first.second].dim);
    m.a = kv.second;
    Sc[kv.first] = std::move(m);
  }
  heis_step(old.sec, cur, Qm, left, J, old.grown, Hc, Sc);
  HeisBlock nb;
  nb.sec = cur;
  nb.grown = true;
  for (auto& kv : Hc) nb.H[kv.first] = std::move(kv.second.a);
  for (auto& kv : Sc) nb.S[kv.first] = std::move(kv.second.a);
  out = std::move(nb);
  return "";
}

std::string heis_side_ops(const OpTable& t, bool left_side, const HeisBlock& b, SideOps& out) {
  const auto& ops = left_side ? t.lops : t.rops;
  out = SideOps();
  out.host_values = true;
  for (int oid = 0; oid < int(ops.size()); ++oid) {
    const BlockOp& op = ops[oid];
    if (op.kind == OP_IDENTITY) continue;
    if (op.kind != OP_MPS_RENORM) return "a Heisenberg block holds only its H and S operators";
    const auto& src = (op.name == "H") ? b.H : b.S;
    for (auto [qo, qi] : allowed(op, b.sec)) {
      add_block(out, oid, qo, qi, b.sec[qo].dim, b.sec[qi].dim);
      auto it = src.find({qo, qi});
      if (it != src.end()) std::copy(it->second.begin(), it->second.end(), &out.arena[out.blocks.back().off]);
    }
  }
  return "";
}

// ------------------------------------------------------------ task table
std::string build_tasks(const OpTable& t, const std::vector<Sector>& left, const std::vector<Sector>& right,
                        const std::vector<Block>& blocks, int twoS, const SideOps& L, const SideOps& R,
                        std::vector<Task>& tasks) {
  std::vector<int> sN, sS;
  site_states(t.site_kind, sN, sS);
  const int ns = int(sN.size());
  std::unordered_map<uint64_t, int> bidx;
  auto bkey = [](int a, int s1, int s2, int b, int j1, int j2) {
    return (uint64_t(a) << 44) | (uint64_t(s1) << 42) | (uint64_t(s2) << 40) | (uint64_t(b) << 24) |
           (uint64_t(j1) << 12) | uint64_t(j2);
  };
  for (int i = 0; i < int(blocks.size()); ++i) {
    const Block& B = blocks[i];
    bidx[bkey(B.a, B.s1, B.s2, B.b, B.jL1, B.j2R)] = i;
  }
  auto outs = [](const BlockOp& op, const std::vector<Sector>& sec, int q) {
    std::vector<int> r;
    if (op.kind == OP_IDENTITY) {
      r.push_back(q);
      return r;
    }
    for (int p = 0; p < int(sec.size()); ++p)
      if (sec[p].N == sec[q].N + op.dN && triangle(sec[q].twoS, op.k, sec[p].twoS)) r.push_back(p);
    return r;
  };
  tasks.clear();
  for (int ti = 0; ti < int(t.terms.size()); ++ti) {
    const Term& term = t.terms[ti];
    const BlockOp& Aop = t.lops[term.A];
    const BlockOp& Dop = t.rops[term.D];
    const int k = term.k;
    for (int e = 0; e < int(blocks.size()); ++e) {
      const Block& E = blocks[e];
      const int Na = left[E.a].N, Sa = left[E.a].twoS, Sb = right[E.b].twoS;
      const int n1 = sN[E.s1], n2 = sN[E.s2], t1 = sS[E.s1], t2 = sS[E.s2];
      const int sexp = term.B.parity * Na + term.C.parity * (Na + n1) + Dop.parity * (Na + n1 + n2);
      const double sign = (sexp % 2) ? -1.0 : 1.0;
      for (int ap : outs(Aop, left, E.a)) {
        const int Sap = left[ap].twoS;
        const int ablk = Aop.kind == OP_IDENTITY ? -1 : L.find(term.A, ap, E.a);
        if (Aop.kind != OP_IDENTITY && ablk < 0) return "missing left operator block";
        for (int s1p = 0; s1p < ns; ++s1p) {
          const double bval = term.B.red[s1p][E.s1];
          if (bval == 0.0) continue;
          for (int s2p = 0; s2p < ns; ++s2p) {
            const double cval = term.C.red[s2p][E.s2];
            if (cval == 0.0) continue;
            for (int bp : outs(Dop, right, E.b)) {
              const int Sbp = right[bp].twoS;
              const int dblk = Dop.kind == OP_IDENTITY ? -1 : R.find(term.D, bp, E.b);
              if (Dop.kind != OP_IDENTITY && dblk < 0) return "missing right operator block";
              for (int jL1p = std::abs(Sap - sS[s1p]); jL1p <= Sap + sS[s1p]; jL1p += 2) {
                if (!triangle(E.jL1, k, jL1p)) continue;
                for (int j2Rp = std::abs(sS[s2p] - Sbp); j2Rp <= sS[s2p] + Sbp; j2Rp += 2) {
                  if (!triangle(E.j2R, k, j2Rp) || !triangle(jL1p, j2Rp, twoS)) continue;
                  auto it = bidx.find(bkey(ap, s1p, s2p, bp, jL1p, j2Rp));
                  if (it == bidx.end()) continue;
                  // sector-value table entry: alpha * B * C * C~_l * C~_r * C~_h * sign
                  const double cl = ctilde(Sa, t1, E.jL1, Aop.k, term.B.k, k, Sap, sS[s1p], jL1p);
                  const double cr = ctilde(t2, Sb, E.j2R, term.C.k, Dop.k, k, sS[s2p], Sbp, j2Rp);
                  const double ch = ctilde(E.jL1, E.j2R, twoS, k, k, 0, jL1p, j2Rp, twoS);
                  Task x;
                  x.f = it->second;
                  x.term = ti;
                  x.e = e;
                  x.ao = Aop.kind == OP_IDENTITY ? -1 : ap;
                  x.ai = Aop.kind == OP_IDENTITY ? -1 : E.a;
                  x.bo = Dop.kind == OP_IDENTITY ? -1 : bp;
                  x.bi = Dop.kind == OP_IDENTITY ? -1 : E.b;
                  x.ablk = ablk;
                  x.dblk = dblk;
                  x.v = term.alpha * bval * cval * cl * cr * ch * sign;
                  tasks.push_back(x);
                }
              }
            }
          }
        }
      }
    }
  }
  std::stable_sort(tasks.begin(), tasks.end(), [](const Task& x, const Task& y) {
    return std::tie(x.f, x.term, x.e) < std::tie(y.f, y.term, y.e);
  });
  return "";
}

// ------------------------------------------------------------ U(1)-expanded flops
// The paper compares SU(2) with U(1) DMRG by the ratio of their flop counts
// (R_CC, Table 1).  Here the same operator-table is expanded into its spin
// components: each row i becomes the products A_qA B_qB C_qC D_qD with a
// non-zero Clebsch-Gordan weight in [[A x B]^k x [C x D]^k]^0, acting on the
// U(1) two-site blocks (N_a, M_a; site m-states; N_b, M_b) of the M = S
// sector, whose bond blocks have dimension sum_{S >= |M|} d_(N,S).  Flops
// follow the SU(2) rules: E D^T once per distinct (right operator, its
// component, input block, output right sector), A T per task, identities
// skipped.
double u1_counted_flops(const OpTable& t, const std::vector<Sector>& left, const std::vector<Sector>& right, int N,
                        int twoS) {
  std::vector<int> sN, sS;
  site_states(t.site_kind, sN, sS);
  auto u1 = [](const std::vector<Sector>& sec) {
    std::map<std::pair<int, int>, int64_t> d;
    for (const Sector& q : sec)
      for (int m = -q.twoS; m <= q.twoS; m += 2) d[{q.N, m}] += q.dim;
    return d;
  };
  const auto dl = u1(left), dr = u1(right);
  struct MS { int s, m; };
  std::vector<MS> ms;
  for (int s = 0; s < int(sN.size()); ++s)
    for (int m = -sS[s]; m <= sS[s]; m += 2) ms.push_back({s, m});
  struct UB { int Na, Ma, i1, i2, Nb, Mb; };
  std::vector<UB> blocks;
  std::map<std::tuple<int, int, int, int, int, int>, int> bidx;
  for (const auto& [a, da] : dl)
    for (int i1 = 0; i1 < int(ms.size()); ++i1)
      for (int i2 = 0; i2 < int(ms.size()); ++i2)
        for (const auto& [b, db] : dr) {
          if (a.first + sN[ms[i1].s] + sN[ms[i2].s] + b.first != N) continue;
          if (a.second + ms[i1].m + ms[i2].m + b.second != twoS) continue;
          bidx[{a.first, a.second, i1, i2, b.first, b.second}] = int(blocks.size());
          blocks.push_back({a.first, a.second, i1, i2, b.first, b.second});
        }
  // site transitions of one component of a site operator
  auto site_next = [&](const SiteOp& op, int i, int q, std::vector<int>& out) {
    out.clear();
    for (int j = 0; j < int(ms.size()); ++j) {
      if (ms[j].m != ms[i].m + q) continue;
      if (op.red[ms[j].s][ms[i].s] == 0.0) continue;
      if (cg_coef(sS[ms[i].s], ms[i].m, op.k, q, sS[ms[j].s], ms[j].m) == 0.0) continue;
      out.push_back(j);
    }
  };
  double flops = 0.0;
  std::set<std::tuple<int, int, int, int, int>> k1seen;
  std::vector<int> n1, n2;
  for (const Term& term : t.terms) {
    const BlockOp& A = t.lops[term.A];
    const BlockOp& D = t.rops[term.D];
    const bool aid = A.kind == OP_IDENTITY, did = D.kind == OP_IDENTITY;
    const int k = term.k;
    for (int q = -k; q <= k; q += 2) {
      const double c0 = cg_coef(k, q, k, -q, 0, 0);
      if (c0 == 0.0) continue;
      for (int qA = -A.k; qA <= A.k; qA += 2) {
        const int qB = q - qA;
        if (std::abs(qB) > term.B.k || cg_coef(A.k, qA, term.B.k, qB, k, q) == 0.0) continue;
        for (int qC = -term.C.k; qC <= term.C.k; qC += 2) {
          const int qD = -q - qC;
          if (std::abs(qD) > D.k || cg_coef(term.C.k, qC, D.k, qD, k, -q) == 0.0) continue;
          for (int e = 0; e < int(blocks.size()); ++e) {
            const UB& E = blocks[e];
            const auto ao = std::make_pair(E.Na + A.dN, E.Ma + qA);
            const auto bo = std::make_pair(E.Nb + D.dN, E.Mb + qD);
            auto ia = dl.find(ao);
            auto ib = dr.find(bo);
            if (ia == dl.end() || ib == dr.end()) continue;
            site_next(term.B, E.i1, qB, n1);
            if (n1.empty()) continue;
            site_next(term.C, E.i2, qC, n2);
            if (n2.empty()) continue;
            const int64_t k1 = dl.at({E.Na, E.Ma}), k2 = dr.at({E.Nb, E.Mb}), m = ia->second, n = ib->second;
            for (int j1 : n1)
              for (int j2 : n2) {
                if (!bidx.count({ao.first, ao.second, j1, j2, bo.first, bo.second})) continue;
                if (!did && k1seen.insert({term.D, qD, bo.first, bo.second, e}).second) flops += 2.0 * k1 * k2 * n;
                if (!aid) flops += 2.0 * m * k1 * n;
              }
          }
        }
      }
    }
  }
  return flops;
}

}  // namespace su2
