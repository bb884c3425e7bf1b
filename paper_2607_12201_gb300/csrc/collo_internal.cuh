// Internal definitions shared by the CUDA translation units of libcollo.
//
// Notation follows the paper's Eq. 2 / Eq. 3: element i = 0..N-1, interpolation
// point j = 0..K, species s, parameter q, h = T / N.  Two collocation schemes:
// Radau IIA with K = 3 (tau_K = 1, continuity weights b_j = delta_jK) and
// Gauss-Legendre with K = 4 (interior roots, b_j = l_j(1)), Eq. 2c.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "collo.h"

namespace collo {

constexpr int KMAX = 4;          // most collocation points per element
constexpr int NPMAX = KMAX + 1;  // most interpolation points per element

// ---- element-local ordering of the KKT unknowns -----------------------------
// The 2 (K+1) n unknowns of element i's block are grouped into K + 1 groups of
// n (state, multiplier) pairs.  Group g pairs state z[i][pt(g)][s] with the
// multiplier of constraint con(g):
//   Radau K = 3:  (z1, c1) (z2, c2) (z0, c3) | (z3, c0)
//   Gauss K = 4:  (z1, c1) (z2, c2) (z3, c3) (z4, c4) | (z0, c0 of element i+1)
// The first K groups are the element interior (eliminated locally); the last
// is the chain group.  Radau: z3 couples forward to the next element's
// continuity row c0 and c0 back to the previous element's z3, so the chain
// block of element i is (z_i3, c_i0).  Gauss: the outgoing continuity row
// c_(i+1)0 = z_(i+1)0 - sum_j b_j z_ij touches every point of element i, so
// it joins element i's block; the chain block of element i is (z_i0, c_i0),
// whose (c_i0, z_i0) entry is the constant identity, and element i's
// condensation writes the z part of chain block i and the c part of chain
// block i + 1.  Local index of the state of pair (g, s) is 2 (g n + s), of the
// multiplier 2 (g n + s) + 1.
__host__ __device__ inline int grp_point(int gauss, int K, int g) {
  if (gauss) return g < K ? g + 1 : 0;
  return g == 0 ? 1 : (g == 1 ? 2 : (g == 2 ? 0 : 3));
}
// constraint point of group g's multiplier; Gauss's chain group holds the
// next element's c0 (returned as K + 1)
__host__ __device__ inline int grp_con(int gauss, int K, int g) {
  if (gauss) return g < K ? g + 1 : K + 1;
  return g == 0 ? 1 : (g == 1 ? 2 : (g == 2 ? 3 : 0));
}

// Plain-old-data view of one problem's device arrays, passed by value.
struct DevProb {
  int n, r, p, N, M;   // N: elements of all conditions (Nc x Nch)
  int Nc, Nch;         // experimental conditions, elements per condition
  int K;        // collocation points per element (3 Radau, 4 Gauss)
  int np;       // K + 1 interpolation points
  int gauss;    // 1: Gauss-Legendre points, 0: Radau IIA
  int cpt;      // point of the chain block's state: K (Radau) or 0 (Gauss)
  int m;        // 2 (K + 1) n: element unknowns
  int ext;      // m + p: element block plus parameter border
  int bext;     // 4 n + p: cyclic-reduction block (2n) + two neighbour slices + border
  int logscale;
  double h, T;
  // collocation tables (kernel-parameter space): tau[j], D[k][j] = l_j'(tau_k),
  // continuity weights bw[j] (Eq. 2c)
  double tau[NPMAX];
  double D[NPMAX][NPMAX];
  double bw[NPMAX];
  // network
  const int* react;      // [r][2]
  const int* prod;       // [r][2]
  const int* pidx;       // [r]
  const double* kfix;    // [r]
  const double* x0;      // [Nc][n] initial state of each condition
  const double* kscale;  // [Nc][r] condition multipliers of the rate constants, or null
  const double* theta_lo, *theta_hi;  // [p]
  // species -> (reaction, stoichiometric coefficient) CSR
  const int* nu_ptr; const int* nu_r; const double* nu_v;
  // species -> reactions consuming it (each reaction listed once) CSR
  const int* rs_ptr; const int* rs_r;
  // parameter -> reactions it drives CSR
  const int* pr_ptr; const int* pr_r;
  // structural nonzeros of the element derivative blocks (entries outside are
  // exactly zero at every point), ascending index lists in CSR form
  const int* jzr_ptr; const int* jzr_i;   // JZ row s -> columns t
  const int* jzc_ptr; const int* jzc_i;   // JZ column s -> rows t
  const int* wzr_ptr; const int* wzr_i;   // Wzz row t -> columns u
  const int* wtr_ptr; const int* wtr_i;   // Wzt row t -> parameters q
  const int* jtr_ptr; const int* jtr_i;   // JT row s -> parameters q
  const int* thq_ptr; const int* thq_i;   // parameter q -> rows s of Wzt or JT
  const int* obs_sp;                       // [n] 1 if species s is observed
  // observations grouped by element: CSR over elements
  const int* obs_ptr;    // [N+1]
  const int* obs_s;      // [M] species
  const double* obs_y;   // [M]
  const double* obs_sig; // [M]
  const double* obs_w;   // [M][K+1] Lagrange weights l_j(tau_m)
};

// Evaluation outputs kept in the problem (FP64).
struct DevEval {
  double* c;        // [N][K+1][n]
  double* grad;     // [n_x]
  double* JZ;       // [N][K][n][n]
  double* JT;       // [N][K][n][p]
  double* Wzz;      // [N][K][n][n]
  double* Wzt;      // [N][K][n][p]
  double* Wobj;     // [N][n][K+1][K+1]
  double* part;     // [N][4] per element: phi, sum|c|, max|c|, unused
  double* wtt_part; // [N][p]
  double* red;      // [8]: phi, |c|_1, |c|_inf, ...
  double* wtt;      // [p]
};

// Grid barrier state of the persistent cooperative kernels (device memory,
// zero-initialised; err != 0 records a barrier that gave up waiting).
struct GridBar {
  unsigned int count;   // arrivals in the current launch
  unsigned int exits;   // blocks that have left the current launch
  int err;
  // arrivals each barrier waits for beyond the grid's own (0; a failure test
  // sets 1 so that no barrier can complete and every wait runs out)
  unsigned int extra;
  long long spin_limit; // polls before a wait gives up (0: GRID_SPIN_LIMIT)
};

// Factorization storage (T = double or float).
template <typename T>
struct DevFactor {
  T* Lel;        // [N][2Kn][ext]  element interior L columns (column-major)
  T* Del;        // [N][Kn][3]     element interior 2x2 pivots (a, b, d)
  T* Aif;        // [N][2n][2n]    chain blocks (full symmetric)
  T* Cpl;        // [N][n][n]      coupling K[c0 of block, chain state of left neighbour]
  T* Bif;        // [N][2n][p]     interface border
  T* Lb;         // [N][2n][bext]  cyclic-reduction L columns
  T* Db;         // [N][n][3]      cyclic-reduction 2x2 pivots
  double* Scon;  // [2N][p][p]     parameter Schur contributions
  int* inert;    // [2N][3]        (pos, neg, zero) per factored block
  T* work;       // global slab workspace for element blocks too large for smem
  int n_slabs;
  // solve vectors
  T* Vint;       // [N][2Kn] D^-1 L^-1 rhs of the interior
  T* Rif;        // [N][2n]  interface rhs (updated through the reduction)
  T* Vb;         // [N][2n]  D^-1 L^-1 rhs of each reduced block
  double* Rth;   // [2N][p]  parameter rhs contributions
  double* chunkS;  // [CHUNKS][p][p] partial sums of Scon
  double* chunkR;  // [CHUNKS][p]    partial sums of Rth
  GridBar* gbar;   // barrier of the persistent kernels
  int persistent;  // 1: persistent cooperative kernels, 0: one launch per level
};

// Deterministic two-stage sums over many per-block contributions: stage 1
// sums fixed chunks of the contribution index in parallel, stage 2 (inside
// the consumer kernel) adds the chunk sums in order.
constexpr int CHUNKS = 64;
__host__ __device__ inline int n_chunks(int C) { return C < CHUNKS ? (C > 0 ? C : 1) : CHUNKS; }

struct DevSchur {
  double* S;       // [p][p] assembled, then overwritten by L (unit lower) and D;
                   // followed by [p] of scratch (schur_doubles), the multiplier
                   // row of the factorization when it runs in global memory
  double* Sd;      // [p] pivots
  double* xth;     // [p] parameter solution
  long long* inertia;  // [3] total inertia
  double* diag;    // [p] W_thth + sigma_theta + delta_w (assembled by host-side launch)
};

// Doubles of DevSchur::S: the p x p block and the p-entry multiplier row the
// factorization uses when the block does not fit in shared memory.
inline size_t schur_doubles(int p) { return (size_t)p * p + (size_t)p; }

// ---- batched execution ------------------------------------------------------------
// Everything one instance owns on the device, gathered for batched kernels.
struct DevInst {
  DevProb P;
  DevEval E;
  DevFactor<float> F32;
  DevFactor<double> F64;
  DevSchur S;
  double* sigma;      // [n_x]
  double* x;          // [n_x] iterate
  double* lam;        // [n_c]
  double* zl, *zu;    // [p]
  double* dz;         // [2p]
  double* bar;        // [p]  mu/sl - mu/su
  double* zlmzu;      // [p]  zl - zu
  double* th0;        // [p]  starting parameters
  double* ka, *kb, *kr, *kc;   // [n_x + n_c] rhs, solution, residual, correction
  double* thpart;     // [N][p]
  double* npart;      // [N][3]
  double* out;        // [64] per-instance scalar outputs of the batched kernels
  int* fails;         // [1]
  float* sweep_work;  // forward-sweep FP32 matrix when Kn is large
  long long n_x, n_c;
};

// Per-instance, per-launch parameters written by the host.
struct InstParams {
  double dw, dc, mu, tau, alpha, alpha_z, ksig, obj_factor;
};

// Slots of DevInst::out
enum OutSlot {
  O_PHI = 0, O_C1 = 1, O_CINF = 2,            // eval reduction
  O_WMAX = 4, O_WMIN = 5, O_ZSUM = 6, O_LOG = 7,  // theta_prep
  O_RX = 8, O_RC = 9, O_BMAX = 10,           // residual norms
  O_LAM1 = 12, O_GDX = 13,                    // |lambda|_1, grad^T dx
  O_AMAX = 16, O_AZ = 17, O_GPHI = 18,        // theta_step
  O_TLOG = 20, O_TOK = 21,                    // trial barrier
  O_INERT = 24,                               // 3 x long long (24..26)
  O_BERR = 28,                                // grid barrier error flag (as double)
};

// Element i starts its condition's chain (its row 0 is an initial condition).
__host__ __device__ inline bool chain_start(const DevProb& P, int i) { return i % P.Nch == 0; }
// Element i has a successor in its chain (whose row 0 is a continuity row).
__host__ __device__ inline bool chain_next(const DevProb& P, int i) {
  return i + 1 < P.N && !chain_start(P, i + 1);
}

// Find k with pre[k] <= t < pre[k+1] (pre[0] = 0, A + 1 entries).
__device__ inline int find_item(const int* __restrict__ pre, int A, int t) {
  int lo = 0, hi = A;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// Launches whose dynamic shared memory exceeds this opt in through
// cudaFuncAttributeMaxDynamicSharedMemorySize.  Without the opt-in a block may
// use 48 KB of static plus dynamic shared memory; the kernels here declare
// at most 32 KB statically, so 16 KB of dynamic memory always fits.
constexpr size_t SMEM_OPTIN_ABOVE = 16 * 1024;
// Dynamic shared memory of a factorization block above which its elimination
// runs in a global slab instead (allocation and use both test against it).
constexpr size_t FACTOR_SMEM_LIMIT = 200 * 1024;

// ---- error handling -----------------------------------------------------------
void set_error(const std::string& msg);
#define COLLO_CUDA(call)                                                         \
  do {                                                                           \
    cudaError_t _e = (call);                                                     \
    if (_e != cudaSuccess) {                                                     \
      ::collo::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));    \
      return COLLO_ERR_DEVICE;                                                   \
    }                                                                            \
  } while (0)

// Count of kernels this library has launched (all threads, all problems).
void count_launch(int k = 1);

// Launch schedule of the batched kernels (process-wide; collo_set_schedule,
// collo_autotune).  Results are bitwise reproducible for a fixed schedule;
// slab_pairs changes the rounding of blocks held in the global slab.
struct Schedule {
  int big_threads = 512;   // large-element kernel: 512 threads x 1 block per SM, or 256 x 2
  int slab_pairs = 16;     // pairs per panel of blocks in the global slab (8 | 16)
  int solve_top = 8;       // the solve's per-instance top levels: at most this many blocks
  int solve_elems = 8;     // elements per 8-warp block of the solve's grid
};
Schedule& schedule();

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace collo
