// Storage and internal entry points of the relaxed-equality ("lifted")
// condensed-space Newton step (lifted.cu), shared with its interior-point
// driver (lifted_ipm.cu).
#pragma once

#include "problem.cuh"

namespace collo {

constexpr int LBS = 256;   // threads of the lifted kernels

// Device view of the lifted factorization (passed to kernels by value).
struct DevLifted {
  int me = 0;          // element block order Kn + 2n + p
  int kn = 0;          // interior unknowns K n
  int grid_e = 0;      // blocks of the element kernels (one per element)
  bool elem_smem = false;   // element blocks factored in shared memory
  int cw = 0;          // right-hand-side columns per pass of the chain eliminations
  int chunks = 0;      // partial sums of the parameter block
  double dw = 0.0;
  double* sigx = nullptr;   // [n_x]
  double* d = nullptr;      // [n_c] Sigma_s + dw
  double* blk = nullptr;    // [N][me (me + 1) / 2] element blocks (packed lower)
  double* Dg = nullptr;     // [N][n][n] chain diagonal blocks, then their Cholesky factors
  double* Cp = nullptr;     // [N][n][n] coupling of chain block i to the next active one
  double* Xa = nullptr;     // [N][n][n] L_j^-1 (coupling to the left neighbour)
  double* Xb = nullptr;     // [N][n][n] L_j^-1 (coupling to the right neighbour)
  double* Bd = nullptr;     // [N][n][p] chain border
  double* Xt = nullptr;     // [N][n][p] L_j^-1 border
  double* S = nullptr;      // [p][p] parameter block, then its Cholesky factor
  double* Spart = nullptr;  // [chunks][p][p] + p: partial sums of the parameter block, of
                            // its right-hand side ([chunks][p]) and the scratch row of its
                            // Cholesky in global memory
  int* flag = nullptr;      // [1] a pivot was not positive
  // solve
  double* rx = nullptr, *rs = nullptr, *rc = nullptr;   // right-hand side
  double* dx = nullptr, *ds = nullptr, *dl = nullptr;   // solution
  double* ex = nullptr, *es = nullptr, *el = nullptr;   // correction
  double* qx = nullptr, *qs = nullptr, *qc = nullptr;   // residual of the unreduced system
  double* y = nullptr;      // [n_x] condensed rhs, then interior forward values
  double* ue = nullptr;     // [N][2n+p] element contributions to the frontal rhs
  double* cc = nullptr;     // [N][n] chain rhs, then w, then the chain solution
  double* ct = nullptr;     // [p] parameter rhs, then its solution
  double* vneg = nullptr;   // [n_c]
  double* res = nullptr;    // [n_x + n_c] output of the structured residual
  double* nrm = nullptr;    // [8] residual norms
};

struct LiftedStore {
  DevArena mem;
  DevLifted V;
  long long eval_count = -1;   // evaluation the factorization belongs to
  bool pd = false;
};

// Allocate the store on the first call (INVALID_ARG when the chain blocks are
// too large for the reduction kernels).
collo_status lifted_storage(collo_problem* pr);
// Factor with sigma_x already in V.sigx and sigma_s (device) copied into V.d
// (may be V.d itself), then d += dw.  *pd: every pivot was positive.
collo_status lifted_factor_dev(collo_problem* pr, const double* sigma_s, double dw, bool* pd);
// Solve with refinement from V.rx / V.rs / V.rc into V.dx / V.ds / V.dl.
collo_status lifted_solve_dev(collo_problem* pr, int refine_max, double refine_tol, int* sweeps,
                              double* rel);
// Blocks of an element-wise kernel of LBS threads over n entries.
int lifted_grid(size_t n);

}  // namespace collo
