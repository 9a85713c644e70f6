/*
 * su2dmrg: GB300 (sm_103a) library for the projected two-site Hamiltonian
 * application H.psi of SU(2) spin-adapted DMRG and the Davidson eigensolver
 * around it (arXiv:2309.16724).
 *
 * Every entry point returns an su2_status; no exception, exit or assert
 * crosses the ABI.  On failure, su2_last_error(ctx) holds a one-line reason.
 * Spins are passed as "twos" (the integer 2j).  All floating-point data is
 * FP64, matrices are column-major.
 *
 * Ownership: handles are created and destroyed by the library.  psi buffers
 * passed to su2_apply_heff / su2_davidson_create are caller-owned device
 * memory of length psi_len doubles (block order of su2_sectors_query).
 * Environments, task tables and workspaces are library-owned device memory.
 * Concurrency: one context per stream; calls on a context are stream
 * ordered; su2_apply_heff does not synchronise the host.
 */
#ifndef SU2DMRG_H
#define SU2DMRG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct su2_ctx su2_ctx;
typedef struct su2_sectors su2_sectors;
typedef struct su2_env su2_env;
typedef struct su2_dav su2_dav;

enum su2_status {
  SU2_OK = 0,        /* success */
  SU2_EINVAL = 1,    /* bad argument: null/misaligned pointer, triangle or
                        particle-number violation, unknown enum value */
  SU2_ENOMEM = 2,    /* host or device allocation failed */
  SU2_ECUDA = 3,     /* a CUDA runtime call failed */
  SU2_ETIMEOUT = 4,  /* a bounded device-side wait gave up */
  SU2_ENOTCONV = 5   /* Davidson reached its iteration limit */
};

/* Arithmetic of the sector GEMMs of H.psi. */
enum su2_prec {
  SU2_FP64 = 0,        /* native FP64 (CUDA-core DFMA)                       */
  SU2_SPLIT_BF16 = 1,  /* FP64 operands cut into BF16 slices, tcgen05 tensor
                          cores with FP32 accumulation, exact per K-chunk,
                          recombined to FP64                                  */
  SU2_SPLIT_FP8 = 2    /* reserved, not built: FP8 E4M3 slices would need
                          about ten slices and 55 slice products per 16 K
                          against 15 for BF16 (slower at twice the rate);
                          every call rejects it with SU2_EINVAL              */
};

enum su2_site_kind { SU2_SITE_SPIN_HALF = 0, SU2_SITE_ORBITAL = 1 };

/* Operator tables (rows of Eq. 2) the library can build. */
enum su2_model {
  SU2_MODEL_HEISENBERG = 0,   /* J sum S_i.S_{i+1}; block operators
                                 renormalised from a seeded MPS (Sec. II.C) */
  SU2_MODEL_QC_SKELETON = 1,  /* ab initio normal/complementary term
                                 structure, seeded synthetic entries         */
  SU2_MODEL_CASIMIR_S2 = 2,   /* total spin squared (S(S+1) psi)            */
  SU2_MODEL_CASIMIR_N = 3,    /* total particle number (N psi)              */
  SU2_MODEL_AB_INITIO = 4     /* H = sum h_ij E_ij + 1/2 sum (ij|kl)(E_ij E_kl
                                 - delta_jk E_il) of Eq. 1 from the caller's
                                 integrals: spin-adapted normal (left block)
                                 and complementary (right block) operators of
                                 Sec. II.A, renormalised orbital by orbital
                                 from a seeded SU(2) MPS (Sec. II.C) on the
                                 context's GPU (Sec. IV.D), or on the host
                                 for a host-only context                     */
};

/* One bond sector: particle number, twice the spin, kept multiplets. */
typedef struct { int32_t N, twoS, dim; } su2_sector;

/* One block of psi (sector-table row, Sec. II.A): left sector a, site
 * states s1, s2, right sector b, intermediate spins (a x s1)->jL1,
 * (s2 x b)->j2R; a rows x cols column-major matrix at element offset. */
typedef struct {
  int32_t a, s1, s2, b, jL1, j2R, rows, cols;
  int64_t offset;
} su2_block;

/* Bond sectors of a block grown site by site: bond k (k sites) holds the
 * sectors sectors[bond_offset[k] .. bond_offset[k+1]), ascending (N, 2S).
 * The last bond is the one adjacent to the two-site window. */
typedef struct {
  int32_t n_bonds;
  const int32_t* bond_offset;   /* n_bonds + 1 entries */
  const su2_sector* sectors;
} su2_bond_chain;

typedef struct {
  int32_t model;      /* su2_model */
  int32_t n_left;     /* orbitals / sites in the left block (>= 1; the ab
                         initio model also takes an empty block, 0)      */
  int32_t n_right;    /* orbitals / sites in the right block (likewise)   */
  double J;           /* Heisenberg coupling                 */
  uint64_t seed;      /* seed of the counter-based generator (SplitMix64)
                         for synthetic entries and MPS tensors */
  const double* h;    /* SU2_MODEL_AB_INITIO: host array of the one-electron
                         integrals h_ij, L x L row-major, L = n_left + 2 +
                         n_right orbitals in chain order (left block, the
                         two sites, right block); read during the call   */
  const double* eri;  /* SU2_MODEL_AB_INITIO: host array of the two-electron
                         integrals (ij|kl) (chemists' notation) at
                         ((i L + j) L + k) L + l; read during the call.
                         Other models: both NULL                          */
  const double* mps_left;   /* SU2_MODEL_AB_INITIO (and mps_right of the
                               Heisenberg sweep), optional host arrays of the
                               MPS tensors that grow the left / right block
                               along its bond chain (NULL: the seeded tensors).
                               Layout: for each step k = 1 .. n of the chain,
                               for each sector q of bond k in order, its
                               tensor as a column-major r0 x d_q matrix.  Its
                               rows stack the (previous-bond sector p, site
                               state s) pairs that couple to q, p outer and s
                               inner (orbital sites s: empty, one electron,
                               two electrons; spin-1/2 sites: one state),
                               each pair d_p rows; N_p + N_s = N_q and the
                               spins obey the triangle rule.  The left block
                               grows by orbital k - 1, the right block by
                               orbital L - k.  The columns should be
                               orthonormal (left- resp. right-canonical
                               blocks): H_eff is then the projection of H onto
                               the MPS basis; the library does not check it.
                               Read during the call; the two-site sweep takes
                               mps_right as its initial right blocks.       */
  const double* mps_right;
} su2_hamiltonian;

typedef struct {
  int64_t t_budget_bytes;  /* device bytes for the intermediate T = E D^T of
                              one term chunk (0: library default)           */
  int32_t n_slices;        /* BF16 slices per operand, 2..6 (0: default 5)  */
  int32_t prepare_split;   /* 1: also build the split-precision arenas      */
  int32_t autotune;        /* 1: build the split arenas with the slice count
                              and stage depth picked by measurement on this
                              environment (n_slices is ignored): the
                              smallest S whose H.psi on a seeded vector
                              differs from the S = 6 result by <= split_tol
                              (relative 2-norm), then the fastest valid
                              stage depth.  Costs about a dozen split H.psi
                              and five slab builds.  Not in the paper.     */
  double split_tol;        /* autotune tolerance (0: 3e-11)                 */
  int32_t shard_rank;      /* term sharding (shard_count > 1): this shard  */
  int32_t shard_count;     /* keeps the tasks of its share of the operator
                              terms (longest-processing-time order of their
                              flops), so its H.psi is a partial F and the
                              shards' results sum to H.psi.  For a
                              multi-rank run with one shard per GPU and a
                              sum-reduction of F.  0 / 0: all terms.  The
                              paper's own distribution is by GPU task
                              queues (Sec. III); this is a data-parallel
                              split of Eq. 2's sum over i.                 */
  int32_t spin_limit;      /* polls of each work-loop mbarrier wait in the
                              split GEMM before the CTA gives up, sets the
                              device status to SU2_ETIMEOUT and returns
                              (0: 2^26, seconds of waiting).  A CTA that
                              gives up still waits the full 2^26 polls for
                              its own bulk copies and MMAs before it frees
                              TMEM and exits.  Small values are for testing
                              the timeout path; the H.psi result of a call
                              that timed out is undefined.                 */
  int64_t resident_bytes;  /* out-of-core operators (Sec. III.E-F): 0 keeps
                              every operator block on the device.  > 0:
                              about this many bytes of FP64 operator blocks
                              stay on the device (at least the blocks read
                              by several term chunks, by the diagonal and
                              by the small-task class, then the blocks of
                              the first chunks); the others lie in pinned
                              host memory, the blocks of each chunk
                              contiguous, and every H.psi copies them chunk
                              by chunk into two device slots on an IO
                              stream of the environment, overlapped with
                              the compute of other chunks (one
                              cudaMemcpyAsync per chunk).  The chunk
                              boundaries then bound both the intermediates
                              and the operator bytes of a chunk by
                              t_budget_bytes (0: a quarter of the free
                              device memory beside resident_bytes, at most
                              16 GiB; 4 GiB on a host context).  With a host
                              context only the plan is made (its numbers
                              in su2_env_info; the host arenas take its
                              layout).  The static-scratch entry point and
                              Davidson graph capture reject such an
                              environment (SU2_EINVAL).                    */
} su2_env_opts;

typedef struct {
  int64_t psi_len, n_blocks, n_terms, n_tasks, n_k1, n_chunks;
  double flops_su2;        /* flops of one H.psi as executed (K1 deduplicated
                              by (D operator, output sector, input block),
                              K2 per task; identities skipped)            */
  double flops_u1_equiv;   /* flops_su2 * R_D, R_D = D_U(1)^eff / D        */
  double r_d;              /* D_U(1)^eff / D of the left bond              */
  double env_bytes;        /* FP64 bytes of all operator blocks            */
  int32_t split_slices;    /* slices of the prepared split path (0: none)  */
  int32_t split_stage_k;   /* 16-K steps per pipeline stage of the split GEMM */
  double split_err_est;    /* autotune: relative difference of the chosen
                              S to S = 6 on the test vector (-1: not
                              measured)                                    */
  int64_t t_chunk_bytes;   /* FP64 bytes of the intermediate T of the
                              largest term chunk (native-FP64 path)        */
  double renorm_flops;     /* SU2_MODEL_AB_INITIO: flops of the products
                              of the renormalisation that built the block
                              operators (0 for the other models)           */
  double flops_u1_counted; /* flops of the same operator-table expanded
                              into (N, S_z) sectors (the U(1) blocks of the
                              M = S two-site space), counted with the same
                              rules as flops_su2: the analogue of the
                              paper's U(1) flop count (Table 1)            */
  double r_cc;             /* flops_u1_counted / flops_su2 (the paper's
                              R_CC); with a sharded environment it divides
                              the full table's count by the shard's flops */
  int64_t resident_bytes;  /* FP64 operator bytes on the device            */
  int64_t streamed_bytes;  /* FP64 operator bytes in pinned host memory,
                              copied to the device once per H.psi (0: all
                              resident)                                    */
  int64_t n_io_chunks;     /* term chunks of the out-of-core plan (0: none) */
} su2_env_info;

typedef struct {
  double tol;          /* residual 2-norm (default 1e-8)        */
  int32_t max_sub;     /* subspace size (default 24, max 32)    */
  int32_t keep;        /* Ritz vectors kept on restart (2)      */
  int32_t max_iter;    /* iteration limit (200)                 */
  int32_t prec;        /* su2_prec of the H.psi inside           */
  int32_t use_graph;   /* 1: capture one iteration (H.psi included) as a
                          CUDA graph on the first step and replay it; the
                          subspace size then lives on the device        */
} su2_dav_opts;

/* Context on CUDA device `device` (-1: host-only context that can build
 * sectors and tables but not run kernels) and stream `cuda_stream`
 * (a cudaStream_t; NULL means the legacy default stream).  All device work
 * of the context is ordered on that stream. */
int su2_ctx_create(int device, void* cuda_stream, su2_ctx** out);
int su2_ctx_destroy(su2_ctx* ctx);
const char* su2_last_error(su2_ctx* ctx);
/* Synchronises the context stream and returns (then clears) the device
 * status word that kernels set instead of trapping: 0 = fine, 4 = a
 * bounded device-side wait gave up (SU2_ETIMEOUT).  The call itself
 * returns SU2_ECUDA if the stream reports an error. */
int su2_ctx_status(su2_ctx* ctx, int32_t* device_status);
/* Host watchdog: polls the context stream (cudaStreamQuery) until its work
 * is done or `timeout_s` seconds have passed (timeout_s < 0: no limit).
 * SU2_ETIMEOUT if the stream is still busy at the limit (the work keeps
 * running; the call may be repeated), SU2_ECUDA if the stream reports an
 * error, otherwise the device status word is read and cleared as in
 * su2_ctx_status and a non-zero word returns SU2_ETIMEOUT.  The paper has no
 * counterpart; failure detection of the library. */
int su2_ctx_wait(su2_ctx* ctx, double timeout_s);

/* Sector-table of psi (Sec. II.A, Eq. 3): all blocks (a, s1, s2, b, jL1,
 * j2R) with N_a + n1 + n2 + N_b = N_target and the couplings a x s1 -> jL1,
 * s2 x b -> j2R, jL1 x j2R -> twoS_target allowed.  Host-only work. */
int su2_build_sectors(su2_ctx* ctx, const su2_sector* left, int32_t n_left,
                      const su2_sector* right, int32_t n_right, int32_t site_kind,
                      int32_t N_target, int32_t twoS_target, su2_sectors** out);
int su2_sectors_query(const su2_sectors* s, int64_t* psi_len, int32_t* n_blocks,
                      const su2_block** blocks);
int su2_sectors_destroy(su2_sectors* s);

/* Operator-table (Eq. 2), block operators A_i / D_i, Clebsch-Gordan-layer
 * coefficients C~ (Eq. a, from 6j/9j of Eqs. A2-A4), sector-task-table
 * (Eq. 3) and sector-value table (Sec. II.C), built once per site.  The
 * chains give the bond sectors grown from the vacuum to the two-site
 * window (their last bonds must equal the sectors' left/right lists).  With
 * a device context the tables and operators are uploaded; the ab initio
 * model renormalises its block operators on the device (its products run
 * through the grouped FP64 kernels; intermediate arenas are allocated and
 * freed during the call).  SU2_EINVAL for a missing integral array or
 * chains whose lengths differ from n_left + 1 / n_right + 1. */
int su2_build_environment(su2_ctx* ctx, const su2_hamiltonian* H,
                          const su2_bond_chain* left_chain, const su2_bond_chain* right_chain,
                          const su2_sectors* sectors, const su2_env_opts* opts, su2_env** out);
int su2_env_query(const su2_env* env, su2_env_info* info);
/* Copies the sector-task-table: 8 int32 per task (f, term, e, a_out, a_in,
 * b_out, b_in, flags) with a_* = -1 for an identity left operator, b_* = -1
 * for an identity right operator, and v per task; arrays of n_tasks rows. */
int su2_env_tasks(const su2_env* env, int32_t* rows8, double* v, int64_t n_tasks);
/* Copies the operator-table (Eq. 2): per row i the left operator id of
 * A_i, the right operator id of D_i (op 0 of a side is its identity),
 * the coupling rank k (twos) and alpha_i; any output pointer may be NULL.
 * Arrays of n_terms entries; SU2_EINVAL if n_terms differs. */
int su2_env_terms(const su2_env* env, int32_t* a_op, int32_t* d_op, int32_t* k, double* alpha, int64_t n_terms);
/* Copies block (out sector qo, in sector qi) of block operator `op` of
 * side 0 (left, A_i) or 1 (right, D_i) into out (rows x cols, column-major).
 * SU2_EINVAL if the operator has no such block or the shape differs. */
int su2_env_operator_block(const su2_env* env, int32_t side, int32_t op, int32_t qo, int32_t qi, double* out,
                           int32_t rows, int32_t cols);
int su2_env_destroy(su2_env* env);

/* F = H_eff psi (Eq. 2 over the sector-task-table).  psi_in, psi_out:
 * device pointers, 8-byte aligned, psi_len doubles, not overlapping.  The
 * call does not synchronise: a bounded device wait that gives up during it
 * is reported by the next su2_ctx_status / su2_ctx_wait (or by a
 * synchronising call), and F is then undefined. */
int su2_apply_heff(su2_ctx* ctx, const su2_env* env, const double* psi_in_dev,
                   double* psi_out_dev, int32_t prec);
/* Same with host buffers: copies psi in, runs, copies F out, synchronises;
 * SU2_ETIMEOUT if a bounded device-side wait gave up during the call. */
int su2_apply_heff_host(su2_ctx* ctx, const su2_env* env, const double* psi_in_host,
                        double* psi_out_host, int32_t prec);
/* H.psi for callers that cannot allocate device memory while they run (a
 * memory pool or arena that owns the device, real-time loops where an
 * allocation could stall or fail).  The paper has no counterpart; this is
 * a deployment variant of the native-FP64 su2_apply_heff.  It calls no
 * cudaMalloc, cudaFree or allocating library routine: the intermediate
 * T = E D^T of each term chunk lives in a fixed 64 MiB device array that
 * every GPU loading the library holds until the process exits.  The caller
 * passes psi_in / psi_out (device, 8-byte aligned, psi_len doubles, not
 * overlapping) and an environment built on the same context; an
 * environment whose largest term chunk needs more than 64 MiB of T is
 * rejected with SU2_EINVAL (build it with t_budget_bytes <= 64 MiB).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device); make that first call before any
 * stream capture.  The cached address belongs to the device's primary
 * context: do not use this entry point on a device after cudaDeviceReset in
 * the same process.  The array is resident on a GPU once the library's device module
 * is loaded there; under CUDA's lazy module loading that load (and the
 * driver's 64 MiB allocation for it) may happen inside the first call on a
 * device, so a caller that must not allocate at all makes one call at
 * start-up.  All calls share the one array: calls that overlap on the
 * GPU (other streams, other threads) race on it; calls ordered on one stream
 * are safe.  The array keeps the last call's contents; nothing in it has to
 * start at zero (every element of T that is read is written first). */
int su2_apply_heff_static_scratch(su2_ctx* ctx, const su2_env* env, const double* psi_in_dev,
                                  double* psi_out_dev);
/* Diagonal of H_eff (Davidson preconditioner) into a device buffer. */
int su2_diag_heff(su2_ctx* ctx, const su2_env* env, double* diag_dev);

/* Davidson eigensolver for the lowest eigenpair of H_eff (the
 * diagonalisation that takes 85-90 % of DMRG time, Sec. II).  One call of
 * su2_davidson_step performs one iteration on the device: H.v, projected
 * matrix update, Rayleigh-Ritz, residual, preconditioned correction and
 * Gram-Schmidt; theta and the residual norm are returned. */
int su2_davidson_create(su2_ctx* ctx, const su2_env* env, const double* psi0_dev,
                        const su2_dav_opts* opts, su2_dav** out);
int su2_davidson_step(su2_ctx* ctx, su2_dav* dav, double* theta, double* resnorm);
/* su2_davidson_step synchronises on every iteration and returns
 * SU2_ETIMEOUT (clearing the device status word) if a bounded device-side
 * wait of that iteration gave up; theta and the residual are then not
 * updated.  Runs steps until ||r|| <= tol or max_iter; SU2_ENOTCONV if not
 * reached. */
int su2_davidson_solve(su2_ctx* ctx, su2_dav* dav, double* theta, double* resnorm,
                       int32_t* iterations);
int su2_energy(const su2_dav* dav, double* E);
/* The energy as an expectation value (a10's check of the Davidson
 * eigenvalue): H.x recomputed on the path `prec` for the current Ritz vector
 * x, *rq = <x|Hx> / <x|x> and, if resnorm is not NULL, *resnorm =
 * ||Hx - rq x|| / ||x||.  Synchronises the context stream; allocates two
 * device vectors of psi_len for the call.  SU2_EINVAL for an unknown
 * precision; the device status word as su2_apply_heff_host. */
int su2_energy_check(su2_ctx* ctx, su2_dav* dav, int32_t prec, double* rq, double* resnorm);
/* Current Ritz vector (unit norm, largest-magnitude entry positive). */
int su2_davidson_vector(su2_ctx* ctx, su2_dav* dav, double* x_dev);
int su2_davidson_destroy(su2_dav* dav);

/* Two-site sweep (Sec. II; target spin S = opts->twoS / 2) of the ab initio model
 * (SU2_MODEL_AB_INITIO with its integrals) or of the spin-1/2 Heisenberg
 * chain (SU2_MODEL_HEISENBERG, coupling J; h and eri unused): at every
 * window (sites i, i+1) the environment is assembled from the blocks of
 * every length the sweep keeps, the lowest eigenpair of H_eff found by
 * Davidson (split or FP64 H.psi), the reduced two-site wavefunction
 * decomposed per bond sector by a singular value decomposition (on the
 * host), the D largest singular values kept (ties to the lower (N, 2S)
 * sector, then the lower index), and the block on the side the sweep moves
 * to grown by one site with the kept singular vectors (ab initio blocks:
 * kept and renormalised on the device, Sec. IV.D; Heisenberg blocks {H, S}:
 * on the host).  The sweep starts at window 0 moving right with the right
 * blocks of a seeded MPS, or of the caller's tensors (H->mps_right), on
 * right_chain (the bonds of 0 .. L-2 sites, L = n_left + 2 + n_right) and
 * turns at the ends.  The first window's Davidson starts from a seeded
 * vector; with `predict` every later window starts from the wavefunction
 * predicted from the previous one (the kept part of its bond matrix expanded
 * over the adjacent block's MPS tensor: the truncated state written in the
 * next window's basis; at a turn, the previous eigenvector), else from a
 * seeded vector too.  Device contexts only. */
typedef struct su2_sweep su2_sweep;
typedef struct {
  int32_t D;             /* multiplets kept per bond                        */
  int32_t prec;          /* su2_prec of the Davidson H.psi                  */
  double tol;            /* Davidson residual 2-norm (0: 1e-8)              */
  int32_t max_iter;      /* Davidson iterations per window (0: 400)         */
  int32_t n_slices;      /* BF16 slices of the split path (0: 5)            */
  uint64_t guess_seed;   /* seed of the Davidson start vectors              */
  int32_t predict;       /* 1: start each window from the predicted vector  */
  int32_t twoS;          /* twice the target spin S (0: singlet)           */
} su2_sweep_opts;
int su2_sweep_create(su2_ctx* ctx, const su2_hamiltonian* H, const su2_bond_chain* right_chain, int32_t N,
                     const su2_sweep_opts* opts, su2_sweep** out);
/* Runs n_steps windows; energies[k] is the Davidson energy of the k-th
 * window run, discarded[k] the weight (sum of sigma^2) dropped by its
 * truncation (0 at a turn), iterations[k] its Davidson iterations and
 * start_energies[k] the Rayleigh quotient of its start vector (the first
 * iteration's Ritz value); any of the four may be NULL. */
int su2_sweep_run(su2_ctx* ctx, su2_sweep* sw, int32_t n_steps, double* energies, double* discarded,
                  int32_t* iterations, double* start_energies);
/* Checkpoint of a sweep that stands at the start of a right-moving
 * half-sweep (before its first window, or after a left-moving half-sweep
 * turned at window 0): the bond chain of its right blocks (bonds of 0 ..
 * L-2 sites, *n_bonds = L - 1) and the MPS tensors that grew them, in the
 * layout of su2_hamiltonian.mps_right.  A sweep created from that chain and
 * those tensors, with the same Hamiltonian, N and options, continues where
 * this one stands (its first window starts from a seeded vector).  With
 * bond_offset, sectors and mps all NULL the call returns the sizes
 * (*n_sectors over all bonds, *n_values doubles); otherwise it fills the
 * caller's arrays, whose capacities the caller passes in *n_bonds (entries
 * of bond_offset minus one), *n_sectors and *n_values.  Host arrays; no
 * device work.  SU2_EINVAL anywhere else in the sweep or for arrays that
 * are too small. */
int su2_sweep_checkpoint(su2_ctx* ctx, su2_sweep* sw, int32_t* n_bonds, int32_t* n_sectors, int64_t* n_values,
                         int32_t* bond_offset, su2_sector* sectors, double* mps);
int su2_sweep_destroy(su2_sweep* sw);

/* Group order of the paper's hash-based semi-dynamic scheduling (Sec.
 * III.D, Fig. 2) for a multi-GPU run: worker `id` of `step` workers picks, at
 * its i-th pick, group (id + step * i + cycle) mod group_count, where
 * cycle = floor(i / cycle_len) and cycle_len = group_count / gcd(group_count,
 * step) is the length of the cyclic subset reached by steps of `step`; the
 * shift by `cycle` makes every group reachable, so group_count consecutive
 * picks visit every group once, and workers start on disjoint groups.
 * Workers claim the tasks of the group they picked from a shared counter (the
 * paper's Contract Book) and move on when it is exhausted.  Host-only
 * arithmetic; SU2_EINVAL unless 0 <= id < step, group_count >= 1, i >= 0. */
int su2_hash_group(int32_t id, int32_t step, int64_t group_count, int64_t i, int64_t* group);

/* Per-kernel timing of su2_apply_heff (off by default): with profiling on,
 * every kernel launch of the hot path is bracketed by CUDA events on the
 * context stream.  su2_profile_read synchronises on the recorded events and
 * returns, for kernel kind `kind` (0: FP64 K1, 1: FP64 K2, 2: split-path
 * kernels other than the GEMMs: slices, exponents, T' slabs and the
 * small-task class, 3: split-path K1, 4: split-path K2), the launches, total
 * device milliseconds and algorithmic flops since the last reset, and the
 * kind's name.  Kind 5 counts every kernel the hot path launched (also with
 * profiling off; no timing).  SU2_EINVAL for an unknown kind. */
int su2_profile_enable(su2_env* env, int32_t on);
int su2_profile_reset(su2_env* env);
int su2_profile_read(su2_env* env, int32_t kind, int64_t* launches, double* ms, double* flops, const char** name);

#ifdef __cplusplus
}
#endif
#endif
