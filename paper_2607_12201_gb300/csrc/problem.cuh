// Host-side problem object of libcollo and the launchers implemented in the
// kernel translation units.
#pragma once

#include <memory>

#include "collo_internal.cuh"

struct collo_problem;

namespace collo {

// launchers (eval.cu)
size_t eval_smem_bytes(const DevProb& P);
cudaError_t launch_obs_weights(const DevProb& P, int M, int N, double T, const double* t,
                               int* elem, double* w, cudaStream_t st);
cudaError_t launch_eval(const DevProb& P, const DevEval& E, const double* x, const double* dx,
                        double alpha, const double* lam, double obj_factor, bool deriv,
                        cudaStream_t st);
cudaError_t launch_kkt_resid(const DevProb& P, const DevEval& E, const double* sigma, double dw,
                             double dc, const double* vx, const double* vl, const double* bx,
                             double bxs, const double* bc, double bcs, double* rout,
                             double* thpart, double* npart, const double* th_extra, double* out,
                             cudaStream_t st);
// launchers (factor.cu)
cudaError_t launch_chunk_sums(const double* X, int C, int L, double* part, cudaStream_t st);
int bcr_levels(int N);
template <typename T>
size_t factor_work_elems(const DevProb& P, int n_slabs);
template <typename T>
cudaError_t launch_elem_factor(const DevProb& P, const DevEval& E, const double* sigma, double dw,
                               double dc, const DevFactor<T>& F, cudaStream_t st);
template <typename T>
cudaError_t launch_factor(const DevProb& P, const DevEval& E, const double* sigma, double dw,
                          double dc, const DevFactor<T>& F, const DevSchur& S, cudaStream_t st);
template <typename T>
cudaError_t launch_solve(const DevProb& P, const DevFactor<T>& F, const DevSchur& S,
                         const double* b, double* sol, cudaStream_t st);

// launchers (ipm.cu)
cudaError_t launch_axpy(double* y, const double* x, double a, size_t n, cudaStream_t st);
cudaError_t launch_forward_sweep(collo_problem* pr);

// Device allocations owned by a problem; freed in the destructor.
struct DevArena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  ~DevArena() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* alloc(size_t count) {
    if (count == 0) count = 1;
    void* p = nullptr;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    bytes += count * sizeof(T);
    return static_cast<T*>(p);
  }
};

template <typename T>
struct FactorStore {
  DevFactor<T> F{};
  bool allocated = false;
};

}  // namespace collo

struct collo_problem;
namespace collo {
collo_status ensure_factor_storage(collo_problem* pr, int precision);
collo_status factor_internal(collo_problem* prob, double dw, double dc, int precision,
                             long long inertia[3]);
collo_status solve_internal(collo_problem* prob, const double* b, double* sol, int refine_max,
                            double refine_tol, int* sweeps, double* resid);
}  // namespace collo

struct collo_problem {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int precision = 0;
  int launch_mode = 0;
  collo::DevProb P{};
  collo::DevEval E{};
  collo::DevSchur S{};
  collo::DevArena arena;
  collo::FactorStore<double> f64;
  collo::FactorStore<float> f32;
  int factored = -1;          // precision of the current factorization, -1 none
  bool evaluated = false;
  int n_slabs = 0;
  // KKT regularisation of the current factorization
  double fac_dw = 0.0, fac_dc = 0.0;
  // device work vectors
  double* sigma = nullptr;    // [n_x]
  double* kvec_a = nullptr;   // [n_x + n_c]  rhs
  double* kvec_b = nullptr;   // [n_x + n_c]  solution
  double* kvec_r = nullptr;   // [n_x + n_c]  residual
  double* kvec_c = nullptr;   // [n_x + n_c]  correction
  double* thpart = nullptr;   // [N][p] then [CHUNKS][p] chunk sums
  double* npart = nullptr;    // [N][2]
  double* scal = nullptr;     // [64] device scalars
  double* red_parts = nullptr;  // [256] partial sums of two-stage reductions
  double* hscal = nullptr;    // [64] pinned host mirror
  // IPM state
  double* x = nullptr;        // [n_x]
  double* lam = nullptr;      // [n_c]
  double* zl = nullptr;       // [p]
  double* zu = nullptr;       // [p]
  double* dz = nullptr;       // [2p] bound-dual steps
  double* thx = nullptr;      // [2p] parameter-space helper vectors
  int* fails = nullptr;       // [1]
  float* sweep_work = nullptr;   // forward-sweep FP32 Newton matrix when too big for smem
  int64_t n_x = 0, n_c = 0;
};
