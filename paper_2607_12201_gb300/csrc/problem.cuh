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

cudaError_t launch_init_point_b(const DevInst* insts, const int* act, int A, double k1, double k2,
                                cudaStream_t st);
cudaError_t launch_sweep_b(const DevInst* insts, const int* act_warp, int A_warp,
                           size_t smem_warp, const int* act_cta, int A_cta, size_t smem_cta,
                           cudaStream_t st);
cudaError_t launch_theta_prep_b(const DevInst* insts, const int* act, int A, const InstParams* prm,
                                cudaStream_t st);
cudaError_t launch_vec_reduce_b(const DevInst* insts, const int* act, int A, int which,
                                cudaStream_t st);
cudaError_t launch_theta_step_b(const DevInst* insts, const int* act, int A, const InstParams* prm,
                                cudaStream_t st);
cudaError_t launch_trial_barrier_b(const DevInst* insts, const int* act, int A,
                                   const InstParams* prm, cudaStream_t st);
cudaError_t launch_update_b(const DevInst* insts, const int* act, int A, const long long* pre,
                            long long total, const InstParams* prm, int mode, cudaStream_t st);
size_t sweep_smem_bytes(const DevProb& P, bool jm_in_smem);
size_t sweep_warp_smem_bytes(const DevProb& P);
// batched launchers (eval.cu, factor.cu); `reserve`: SMs the cooperative
// grids leave to kernels of another stream
cudaError_t launch_eval_b(const DevInst* insts, const int* act, int A, const int* pre_elem,
                          int total_elems, const InstParams* prm, int xsel, int dxsel, int lsel,
                          bool deriv, size_t smem, cudaStream_t st);
cudaError_t launch_resid_b(const DevInst* insts, const int* act, int A, const int* pre_elem,
                           int total_elems, int max_n, const InstParams* prm, int mode,
                           cudaStream_t st);
template <typename T>
cudaError_t launch_factor_b(const DevInst* insts, const int* act, int A, const int* pre_elem,
                            const int* pre_lv, int maxL, const int* pre_cs,
                            const InstParams* prm, const int* flags, GridBar* gb, size_t smem,
                            int grid_cap, int rt_threads, size_t rt_smem, int tot_elem,
                            int big_grid, size_t big_smem, int bcr_tpt, int bcr_full, int parts,
                            cudaStream_t st, int reserve = 0);
// Block size of the register-tiled element condensation for P (0: the
// element does not fit it).
int elem_rt_threads(const DevProb& P, bool f32);
// Tiles per thread of the register-tiled cyclic-reduction blocks (0: none).
int bcr_rt_tiles_of(const DevProb& P);
// Dynamic shared memory of the register-tiled element kernel for P.
size_t elem_rt_stage_bytes(const DevProb& P, bool f32);
// Dynamic shared memory of the register-tiled reduction blocks (both halves of
// a block, two stage buffers per half).
size_t bcr_rt_stage_bytes(const DevProb& P, bool f32);
template <typename T>
cudaError_t launch_solve_b(const DevInst* insts, const int* act, int A, const int* pre_elem,
                           const int* pre_lv, int maxL, int lsplit, const int* pre_cs, int ir,
                           int per_warp,
                           GridBar* gb, int max_p, int grid_want, cudaStream_t st,
                           int reserve = 0);
template <typename T>
size_t elem_factor_smem(const DevProb& P, bool full);
template <typename T>
size_t bcr_factor_smem(const DevProb& P, bool full);

// Device allocations owned by a problem; freed in the destructor (or by
// release).  With `stream` set the allocations are stream-ordered
// (cudaMallocAsync from the device's default pool) and release() returns them
// in stream order, so freeing a store does not synchronise the device.
struct DevArena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  DevArena() = default;
  DevArena(const DevArena&) = delete;
  DevArena& operator=(const DevArena&) = delete;
  DevArena(DevArena&& o) noexcept : ptrs(std::move(o.ptrs)), bytes(o.bytes), stream(o.stream) {
    o.ptrs.clear();
    o.bytes = 0;
  }
  DevArena& operator=(DevArena&& o) noexcept {
    if (this != &o) {
      release(nullptr);
      ptrs = std::move(o.ptrs);
      bytes = o.bytes;
      stream = o.stream;
      o.ptrs.clear();
      o.bytes = 0;
    }
    return *this;
  }
  ~DevArena() { release(nullptr); }
  // Free everything: in stream order on `st` when given, else at once.
  void release(cudaStream_t st) {
    for (void* p : ptrs) {
      if (st) cudaFreeAsync(p, st);
      else cudaFree(p);
    }
    ptrs.clear();
    bytes = 0;
  }
  // Bytes alloc<T>(count) takes.
  template <typename T>
  static size_t bytes_of(size_t count) { return (count ? count : 1) * sizeof(T); }
  template <typename T>
  T* alloc(size_t count) {
    const size_t b = bytes_of<T>(count);
    void* p = nullptr;
    const cudaError_t e = stream ? cudaMallocAsync(&p, b, stream) : cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    bytes += b;
    return static_cast<T*>(p);
  }
};

template <typename T>
struct FactorStore {
  DevFactor<T> F{};
  bool allocated = false;
  DevArena mem;   // this store's arrays (stream-ordered, freed on release)
};

}  // namespace collo

struct collo_problem;
namespace collo {
// Storage of the relaxed-equality (lifted) condensed factorization (lifted.cu).
struct LiftedStore;
void lifted_free(LiftedStore* L);
collo_status lifted_time_launch(collo_problem* pr, int which);
// Host copies of a problem's inputs (for re-creating it on another mesh).
struct HostInputs {
  std::vector<int> react, prod, pidx, species, observable, obs_cond;
  std::vector<double> kfix, x0, lo, hi, t, y, sigma, cond_x0, cond_scale;
  int n_conditions = 1;
};
collo_status ensure_factor_storage(collo_problem* pr, int precision);
// Spare storage of `precision` (and the spare Schur block); swap_spare
// exchanges the primary and spare factorization of `precision` together with
// the Schur blocks.
collo_status ensure_spare_storage(collo_problem* pr, int precision);
void swap_spare(collo_problem* pr, int precision);
// Device bytes the problem holds now (its own arrays and every allocated
// factorization store).
int64_t problem_held_bytes(const collo_problem* pr);
// Device bytes the problem will hold while an interior-point solve in
// `precision` runs on it (the stores ensure_factor_storage and
// ensure_spare_storage add are counted exactly as they would be allocated).
int64_t problem_solve_bytes(const collo_problem* pr, int precision);
// Free every factorization store (stream-ordered on `st`); the problem keeps
// its data, iterate and evaluation arrays and becomes unfactored.
void release_factor_storage(collo_problem* pr, cudaStream_t st);
collo_status factor_internal(collo_problem* prob, double dw, double dc, int precision,
                             long long inertia[3]);
collo_status solve_internal(collo_problem* prob, const double* b, double* sol, int refine_max,
                            double refine_tol, int* sweeps, double* resid);
collo_status runner_eval(collo_problem* pr, double obj_factor);
collo_status runner_time_phase(collo_problem* pr, int phase, int prec, int reps, double* ms);
collo_status runner_factor(collo_problem* pr, int prec, double dw, double dc, long long inertia[3]);
collo_status runner_solve(collo_problem* pr, int refine_max, double refine_tol, int* sweeps,
                          double* resid);
}  // namespace collo

namespace collo {
struct Runner;
}

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
  // spare factorization and Schur storage: the second candidate of a
  // speculative inertia-correction round is factored here (swapped with the
  // primary storage when it is the one chosen)
  collo::FactorStore<double> f64_spare;
  collo::FactorStore<float> f32_spare;
  collo::DevSchur S_spare{};
  bool spare_S = false;
  // evaluation outputs of a second line-search trial (constraints, element
  // partials, reduction), written by trial evaluations in the shadow slot
  double* c_spare = nullptr;
  double* part_spare = nullptr;
  double* red_spare = nullptr;
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
  double* npart = nullptr;    // [N][3]
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
  // grid-barrier wait settings of this problem's own runner
  // (collo_problem_set_wait_limit): polls before a wait gives up (0: default)
  // and the failure-test switch that makes every barrier unreachable
  long long wait_polls = 0;
  int wait_unreachable = 0;
  // inputs as given (collo_problem_create_refined)
  collo::HostInputs host;
  // warm start of the next solve (collo_problem_set_start): states and theta,
  // multipliers
  bool has_start = false;
  double* start_x = nullptr;   // [n_x]
  double* start_lam = nullptr; // [n_c]
  double* refine_buf = nullptr;  // [N + 8] defects and their maximum
  // evaluations with derivatives so far (a factorization records the one it used)
  long long eval_count = 0;
  // lifted condensed factorization (collo_lifted_factor), allocated on first use
  collo::LiftedStore* lifted = nullptr;
  collo::DevInst inst{};            // this problem's device pointers (host copy)
  collo::Runner* self = nullptr;    // single-instance runner (batch of one)
  ~collo_problem();
};
