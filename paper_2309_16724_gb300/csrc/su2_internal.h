// Internal data structures of the su2dmrg library (host side).
#pragma once
#include <cstdint>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "su2dmrg.h"

namespace su2 {

// ---------------------------------------------------------------- coupling
// Wigner 6j by Racah's formula (Eq. A3 with the triangle coefficient of
// Eq. A4), exact in prime-exponent / 128-bit integer arithmetic with one
// final square root; 9j as the x-sum of three 6j (Eq. A2); the scalar
// factor C~ of Eq. a.  Twos arguments.
bool triangle(int a, int b, int c);
double sixj(int a, int b, int c, int d, int e, int f);
double ninej(int j1, int j2, int j, int k1, int k2, int k, int j1p, int j2p, int jp);
double ctilde(int j1, int j2, int j, int k1, int k2, int k, int j1p, int j2p, int jp);
// Clebsch-Gordan coefficient <j1 m1; j2 m2 | J M> (Racah's closed form, twos)
double cg_coef(int j1, int m1, int j2, int m2, int J, int M);

// ---------------------------------------------------------------- model
struct SiteOp {
  int k = 0, dN = 0, parity = 0, n = 1;  // rank (twos), particle change, fermion parity, states
  double red[3][3] = {{0}};               // reduced matrix [out][in], CG form of Wigner-Eckart
};

enum OpKind { OP_IDENTITY = 0, OP_HAM, OP_RANDOM, OP_ADJOINT, OP_MPS_RENORM, OP_SPINTOT, OP_NUMTOT, OP_VALUES };

struct BlockOp {
  std::string name;
  int k = 0, dN = 0, parity = 0, kind = OP_IDENTITY, base = -1;
};

struct Term {
  double alpha = 1.0;
  int A = 0, D = 0, k = 0;  // left op, right op, coupling rank (twos)
  SiteOp B, C;
};

struct OpTable {
  int site_kind = 0;
  std::vector<BlockOp> lops, rops;
  std::vector<Term> terms;
};

struct Sector { int N, twoS, dim; };
struct Block { int a, s1, s2, b, jL1, j2R, rows, cols; int64_t offset; };

void site_states(int site_kind, std::vector<int>& N, std::vector<int>& twoS);
SiteOp site_op(int site_kind, const char* name);
SiteOp site_adjoint(const SiteOp& op, int site_kind);
OpTable make_table(const su2_hamiltonian& H, int site_kind);
// Q factor (positive diagonal of R) of a rows x cols column-major matrix
void orthonormalize(std::vector<double>& G, int rows, int cols);
// the seeded MPS tensor of sector qo at growth step `step` (side 2: left
// blocks, 3: right blocks): the Q factor of the counter-generated r0 x d
// matrix keyed by (seed, side, step, qo)
std::vector<double> seeded_mps_tensor(uint64_t seed, uint64_t side, int step, int qo, int r0, int d);

// ---------------------------------------------------------------- operators
struct OpBlock { int op, qo, qi, rows, cols; int64_t off; };
// block of a synthetic operator generated on the device (counter-based
// SplitMix64 entries; HAM = 0.1 (X + X^T) + diag(2r/d); ADJOINT from its base)
struct GenBlock {
  int64_t off;
  int32_t rows, cols, kind, base_kind;  // kind: 0 random, 1 HAM, 2 adjoint (of a base block of base_kind)
  uint64_t key;                         // the block's key (adjoint: its base block's key)
  double scale;                         // 1/sqrt(max(rows, cols)) or the adjoint factor
  double base_scale;                    // adjoint: the base block's scale
};

struct SideOps {
  std::vector<OpBlock> blocks;
  std::vector<double> arena;  // all blocks, column-major, 2-double aligned (host mode)
  int64_t arena_size = 0;     // doubles
  bool host_values = true;
  std::vector<GenBlock> gen;  // device-generated blocks (device mode)
  double* dev_ready = nullptr;  // device arena already filled by the builder (device mode; the environment takes it)
  std::unordered_map<uint64_t, int> index;  // key(op, qo, qi) -> block
  static uint64_t key(int op, int qo, int qi) {
    return (uint64_t(uint32_t(op)) << 32) | (uint64_t(uint32_t(qo)) << 16) | uint64_t(uint32_t(qi));
  }
  int find(int op, int qo, int qi) const {
    auto it = index.find(key(op, qo, qi));
    return it == index.end() ? -1 : it->second;
  }
};

struct Task {
  int32_t f, term, e, ao, ai, bo, bi;
  int32_t ablk, dblk;  // operator block indices (-1: identity)
  double v;
};

// builds; return empty string on success, else the error message
std::string build_blocks(const std::vector<Sector>& left, const std::vector<Sector>& right, int site_kind,
                         int N, int twoS, std::vector<Block>& blocks, int64_t& psi_len);
std::string build_side_ops(const OpTable& t, bool left_side, const std::vector<std::vector<Sector>>& chain,
                           const su2_hamiltonian& H, SideOps& out, bool host_values = true);
std::string build_tasks(const OpTable& t, const std::vector<Sector>& left, const std::vector<Sector>& right,
                        const std::vector<Block>& blocks, int twoS, const SideOps& L, const SideOps& R,
                        std::vector<Task>& tasks);

// ab initio environment (Eq. 1 from integrals): operator-table and block
// operators of both sides, renormalised on the context's device (device >= 0)
// or on the host
std::string build_abinitio(const su2_hamiltonian& H, const std::vector<std::vector<Sector>>& lchain,
                           const std::vector<std::vector<Sector>>& rchain, int device, void* stream,
                           int64_t t_budget_bytes, OpTable& table, SideOps& L, SideOps& R, double* renorm_flops);

// flops of the same operator-table and task rules expanded into (N, S_z)
// sectors (U(1) blocks of dimension sum_{S >= |M|} d_(N,S)), in the M = S
// sector of the two-site space
double u1_counted_flops(const OpTable& t, const std::vector<Sector>& left, const std::vector<Sector>& right, int N,
                        int twoS);

// Heisenberg block (spin-1/2 sites): its bond sectors and the reduced blocks
// (qo, qi) of H and of the edge spin S, column-major; grown = false for the
// empty block (no operators)
struct HeisBlock {
  std::vector<Sector> sec{Sector{0, 0, 1}};
  std::map<std::pair<int, int>, std::vector<double>> H, S;
  bool grown = false;
};
// one growth step by a site (left: [block x site]; right: [site x block])
// with the MPS tensor Q (per sector of `cur`, stacked rows x dim)
std::string heis_grow(const HeisBlock& old, const std::vector<Sector>& cur, const std::vector<std::vector<double>>& Q,
                      bool left, double J, HeisBlock& out);
// the operators of the Heisenberg table on one side from a block (host values)
std::string heis_side_ops(const OpTable& t, bool left_side, const HeisBlock& b, SideOps& out);

// two-site sweep of the ab initio model (device contexts): blocks of every
// length kept on the device; the environment at window i (sites i, i+1);
// the per-sector SVD of an S = 0 two-site wavefunction with truncation to D
// multiplets; the block grown by one orbital with the kept singular vectors
struct SweepBlocks;
SweepBlocks* sweep_init(const su2_hamiltonian& H, const std::vector<std::vector<Sector>>& rchain, int device,
                        void* stream, int64_t budget, std::string& err);
void sweep_free(SweepBlocks* w);
std::string sweep_env(SweepBlocks* w, int i, OpTable& table, SideOps& L, SideOps& R, std::vector<Sector>& lsec,
                      std::vector<Sector>& rsec);
std::string sweep_split(const std::vector<Block>& blocks, const double* psi, const std::vector<Sector>& lsec,
                        const std::vector<Sector>& rsec, int N, int D, bool left, std::vector<Sector>& new_sec,
                        std::vector<std::vector<double>>& Q, double* discarded,
                        std::vector<std::vector<double>>* rest = nullptr, int site_kind = SU2_SITE_ORBITAL,
                        int twoS = 0);
std::string sweep_grow(SweepBlocks* w, int i, bool left, const std::vector<Sector>& cur,
                       const std::vector<std::vector<double>>& Q);
// the bonds of the right blocks (0 .. L-2 orbitals) and the MPS tensors
// that grew them (tensors[0] empty), for a checkpoint of the sweep
std::string sweep_right_state(SweepBlocks* w, std::vector<std::vector<Sector>>& chain,
                              std::vector<std::vector<std::vector<double>>>& tensors);
// start vector of the next window (i+1 when `right`, else i-1) predicted
// from window i's kept wavefunction (`rest` of sweep_split, after sweep_grow)
std::string sweep_predict(SweepBlocks* w, int i, bool right, const std::vector<Sector>& lsec,
                          const std::vector<Sector>& rsec, int N, const std::vector<Sector>& cur,
                          const std::vector<std::vector<double>>& rest, std::vector<double>& guess, int twoS = 0);
// the same from explicit data: the next window's bond sectors (nl, nr) and
// the MPS tensor T of the block adjacent to window i on the side the sweep
// moves to (its right block moving right, its left block moving left)
std::string predict_guess(bool right, const std::vector<Sector>& lsec, const std::vector<Sector>& rsec,
                          const std::vector<Sector>& nl, const std::vector<Sector>& nr,
                          const std::vector<std::vector<double>>& T, int N, int site_kind,
                          const std::vector<Sector>& cur, const std::vector<std::vector<double>>& rest,
                          std::vector<double>& guess, int twoS = 0);

// counter-based generator (SplitMix64, Steele/Lea/Flood 2014)
uint64_t splitmix(uint64_t x);
uint64_t block_key(uint64_t seed, uint64_t side, uint64_t op, uint64_t qo, uint64_t qi);
double uniform_elem(uint64_t key, uint64_t idx);

}  // namespace su2
