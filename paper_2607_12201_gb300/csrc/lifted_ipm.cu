// Interior-point driver of the relaxed-equality ("lifted") form: the same
// filter line-search method as the augmented driver (Waechter & Biegler 2006;
// paper Introduction, MadNLP), with the relaxed constraints' slacks s and their
// bound duals v_l, v_u as additional bounded variables (-r <= s <= r).
//
// Per iteration, all vectors on the device:
//   evaluation with derivatives; scaled optimality error from one reduction
//   (dual rows of x and s, c(x) - s, complementarity of the four bound
//   families, the 1-norms of the scaling, ||c(x) - s||_1 and the barrier's
//   log sum); barrier update on the host from those scalars; Sigma_x,
//   Sigma_s and the right-hand sides; the lifted factorization with the dw
//   schedule of the inertia correction (a non-positive pivot means the wrong
//   inertia); the refined lifted solve; bound-dual steps, fraction to the
//   boundary and the barrier's directional derivative from one reduction;
//   backtracking trials (evaluation at x + alpha dx, then ||c - s_t||_1 and
//   the log sum at the trial point); the update with the bound-dual reset.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lifted.cuh"
#include "resid.cuh"

namespace collo {

namespace {

constexpr int IBS = 1024;   // threads of the single-block reductions

// Device state of the lifted solve (x, lambda and the theta bound duals are
// the problem's own iterate arrays).
struct DevLiftedIpm {
  double r;          // relaxation
  double* s;         // [n_c] slacks
  double* vl, *vu;   // [n_c] slack bound duals
  double* dvl, *dvu; // [n_c]
  double* dzl, *dzu; // [p]
  double* ss;        // [n_c] Sigma_s
  double* gneg;      // [n_x + n_c] -(grad + J^T lambda) in the first n_x
  double* th;        // [p] pushed theta0
  double* red;       // [16] reduction results
};

__device__ inline double push_lo(double lo, double hi) {
  return lo + fmin(1e-2 * fmax(1.0, fabs(lo)), 1e-2 * (hi - lo));
}
__device__ inline double push_hi(double lo, double hi) {
  return hi - fmin(1e-2 * fmax(1.0, fabs(hi)), 1e-2 * (hi - lo));
}

// theta0 pushed into its bounds (bound_push = bound_frac = 1e-2).
__global__ void k_lip_theta(DevProb P, DevLiftedIpm I, const double* __restrict__ th0) {
  for (int q = threadIdx.x; q < P.p; q += blockDim.x) {
    const double lo = P.theta_lo[q], hi = P.theta_hi[q];
    I.th[q] = fmin(fmax(th0[q], push_lo(lo, hi)), push_hi(lo, hi));
  }
}

// Slacks c(x0) pushed into [-r, r], unit bound duals, lambda = 0.
__global__ void __launch_bounds__(256) k_lip_start(DevProb P, DevEval E, DevLiftedIpm I,
                                                   double* __restrict__ lam,
                                                   double* __restrict__ zl,
                                                   double* __restrict__ zu, size_t nc) {
  const double a = push_lo(-I.r, I.r), b = push_hi(-I.r, I.r);
  const size_t n_all = nc > (size_t)P.p ? nc : (size_t)P.p;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n_all;
       j += (size_t)gridDim.x * blockDim.x) {
    if (j < nc) {
      I.s[j] = fmin(fmax(E.c[j], a), b);
      I.vl[j] = 1.0;
      I.vu[j] = 1.0;
      lam[j] = 0.0;
    }
    if (j < (size_t)P.p) { zl[j] = 1.0; zu[j] = 1.0; }
  }
}

// One-block reduction of the optimality measures at the current iterate:
// red[0] max |dual| (x and s rows), red[1] max |c - s|, red[2] |lambda|_1,
// red[3] |zl|_1 + |zu|_1 + |vl|_1 + |vu|_1, red[4] / red[5] max / min of the
// complementarity products, red[6] ||c - s||_1, red[7] the barrier's log sum.
__global__ void __launch_bounds__(IBS) k_lip_measures(DevProb P, DevEval E, DevLiftedIpm I,
                                                      const double* __restrict__ x,
                                                      const double* __restrict__ lam,
                                                      const double* __restrict__ zl,
                                                      const double* __restrict__ zu, size_t nz,
                                                      size_t nc) {
  __shared__ double sh[IBS];
  const int tid = threadIdx.x;
  const double r = I.r;
  double dmax = 0.0, pmax = 0.0, l1 = 0.0, z1 = 0.0, cmax = -INFINITY, cmin = INFINITY,
         th1 = 0.0, lg = 0.0;
  for (size_t j = tid; j < nz; j += IBS) dmax = fmax(dmax, fabs(I.gneg[j]));
  for (int q = tid; q < P.p; q += IBS) {
    const double t = x[nz + q], sl = t - P.theta_lo[q], su = P.theta_hi[q] - t;
    dmax = fmax(dmax, fabs(-I.gneg[nz + q] - zl[q] + zu[q]));
    z1 += fabs(zl[q]) + fabs(zu[q]);
    const double a = sl * zl[q], b = su * zu[q];
    cmax = fmax(cmax, fmax(a, b));
    cmin = fmin(cmin, fmin(a, b));
    lg += log(sl) + log(su);
  }
  for (size_t j = tid; j < nc; j += IBS) {
    const double s = I.s[j], cs = E.c[j] - s;
    dmax = fmax(dmax, fabs(-lam[j] - I.vl[j] + I.vu[j]));
    pmax = fmax(pmax, fabs(cs));
    th1 += fabs(cs);
    l1 += fabs(lam[j]);
    z1 += fabs(I.vl[j]) + fabs(I.vu[j]);
    const double a = (s + r) * I.vl[j], b = (r - s) * I.vu[j];
    cmax = fmax(cmax, fmax(a, b));
    cmin = fmin(cmin, fmin(a, b));
    lg += log(s + r) + log(r - s);
  }
  dmax = block_max<IBS>(dmax, sh);
  pmax = block_max<IBS>(pmax, sh);
  l1 = block_sum<IBS>(l1, sh);
  z1 = block_sum<IBS>(z1, sh);
  cmax = block_max<IBS>(cmax, sh);
  cmin = -block_max<IBS>(-cmin, sh);
  th1 = block_sum<IBS>(th1, sh);
  lg = block_sum<IBS>(lg, sh);
  if (tid == 0) {
    I.red[0] = dmax; I.red[1] = pmax; I.red[2] = l1; I.red[3] = z1;
    I.red[4] = cmax; I.red[5] = cmin; I.red[6] = th1; I.red[7] = lg;
  }
}

// Sigma_x, Sigma_s and the right-hand sides of the lifted system at barrier mu.
__global__ void __launch_bounds__(256) k_lip_rhs(DevProb P, DevEval E, DevLiftedIpm I,
                                                 DevLifted L, const double* __restrict__ x,
                                                 const double* __restrict__ lam,
                                                 const double* __restrict__ zl,
                                                 const double* __restrict__ zu, double mu,
                                                 size_t nz, size_t nc) {
  const double r = I.r;
  const size_t nx = nz + P.p;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < nx + nc;
       j += (size_t)gridDim.x * blockDim.x) {
    if (j < nz) {
      L.sigx[j] = 0.0;
      L.rx[j] = I.gneg[j];
    } else if (j < nx) {
      const int q = (int)(j - nz);
      const double t = x[j], sl = t - P.theta_lo[q], su = P.theta_hi[q] - t;
      L.sigx[j] = zl[q] / sl + zu[q] / su;
      L.rx[j] = I.gneg[j] + mu / sl - mu / su;
    } else {
      const size_t k = j - nx;
      const double s = I.s[k], a = s + r, b = r - s;
      I.ss[k] = I.vl[k] / a + I.vu[k] / b;
      L.rs[k] = mu / a - mu / b + lam[k];
      L.rc[k] = s - E.c[k];
    }
  }
}

__device__ inline double ftb(double v, double dv, double tau) {
  return dv < 0.0 ? -tau * v / dv : INFINITY;
}

// Bound-dual steps, fraction to the boundary and the barrier's directional
// derivative (one block): red[8] alpha_max, red[9] alpha_z, red[10] gphi.
__global__ void __launch_bounds__(IBS) k_lip_direction(DevProb P, DevEval E, DevLiftedIpm I,
                                                       DevLifted L, const double* __restrict__ x,
                                                       const double* __restrict__ zl,
                                                       const double* __restrict__ zu, double mu,
                                                       double tau, size_t nz, size_t nc) {
  __shared__ double sh[IBS];
  const int tid = threadIdx.x;
  const double r = I.r;
  double amax = INFINITY, az = INFINITY, g = 0.0;
  for (size_t j = tid; j < nz; j += IBS) g += E.grad[j] * L.dx[j];
  for (int q = tid; q < P.p; q += IBS) {
    const double t = x[nz + q], sl = t - P.theta_lo[q], su = P.theta_hi[q] - t;
    const double d = L.dx[nz + q];
    const double dzl = mu / sl - zl[q] - (zl[q] / sl) * d;
    const double dzu = mu / su - zu[q] + (zu[q] / su) * d;
    I.dzl[q] = dzl;
    I.dzu[q] = dzu;
    amax = fmin(amax, fmin(ftb(sl, d, tau), ftb(su, -d, tau)));
    az = fmin(az, fmin(ftb(zl[q], dzl, tau), ftb(zu[q], dzu, tau)));
    g += E.grad[nz + q] * d + (-mu / sl + mu / su) * d;
  }
  for (size_t j = tid; j < nc; j += IBS) {
    const double s = I.s[j], a = s + r, b = r - s, d = L.ds[j];
    const double dvl = mu / a - I.vl[j] - (I.vl[j] / a) * d;
    const double dvu = mu / b - I.vu[j] + (I.vu[j] / b) * d;
    I.dvl[j] = dvl;
    I.dvu[j] = dvu;
    amax = fmin(amax, fmin(ftb(a, d, tau), ftb(b, -d, tau)));
    az = fmin(az, fmin(ftb(I.vl[j], dvl, tau), ftb(I.vu[j], dvu, tau)));
    g += (-mu / a + mu / b) * d;
  }
  amax = -block_max<IBS>(-amax, sh);
  az = -block_max<IBS>(-az, sh);
  g = block_sum<IBS>(g, sh);
  if (tid == 0) {
    I.red[8] = fmin(1.0, amax);
    I.red[9] = fmin(1.0, az);
    I.red[10] = g;
  }
}

// At the trial point x + alpha dx, s + alpha ds (after its evaluation):
// red[11] ||c - s_t||_1, red[12] the barrier's log sum.
__global__ void __launch_bounds__(IBS) k_lip_trial(DevProb P, DevEval E, DevLiftedIpm I,
                                                   DevLifted L, const double* __restrict__ x,
                                                   double alpha, size_t nz, size_t nc) {
  __shared__ double sh[IBS];
  const int tid = threadIdx.x;
  const double r = I.r;
  double th1 = 0.0, lg = 0.0;
  for (int q = tid; q < P.p; q += IBS) {
    const double t = x[nz + q] + alpha * L.dx[nz + q];
    lg += log(t - P.theta_lo[q]) + log(P.theta_hi[q] - t);
  }
  for (size_t j = tid; j < nc; j += IBS) {
    const double st = I.s[j] + alpha * L.ds[j];
    th1 += fabs(E.c[j] - st);
    lg += log(st + r) + log(r - st);
  }
  th1 = block_sum<IBS>(th1, sh);
  lg = block_sum<IBS>(lg, sh);
  if (tid == 0) { I.red[11] = th1; I.red[12] = lg; }
}

// Accepted step and the bound-dual safeguard (Waechter & Biegler 2006, Eq. 16).
__global__ void __launch_bounds__(256) k_lip_update(DevProb P, DevLiftedIpm I, DevLifted L,
                                                    double* __restrict__ x,
                                                    double* __restrict__ lam,
                                                    double* __restrict__ zl,
                                                    double* __restrict__ zu, double alpha,
                                                    double alpha_z, double mu, double ks,
                                                    size_t nz, size_t nc) {
  const double r = I.r;
  const size_t nx = nz + P.p;
  auto reset = [&](double z, double sl) { return fmax(fmin(z, ks * mu / sl), mu / (ks * sl)); };
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < nx + nc;
       j += (size_t)gridDim.x * blockDim.x) {
    if (j < nz) {
      x[j] += alpha * L.dx[j];
    } else if (j < nx) {
      const int q = (int)(j - nz);
      const double t = x[j] + alpha * L.dx[j];
      x[j] = t;
      const double sl = t - P.theta_lo[q], su = P.theta_hi[q] - t;
      zl[q] = reset(zl[q] + alpha_z * I.dzl[q], sl);
      zu[q] = reset(zu[q] + alpha_z * I.dzu[q], su);
    } else {
      const size_t k = j - nx;
      const double s = I.s[k] + alpha * L.ds[k];
      I.s[k] = s;
      lam[k] += alpha * L.dl[k];
      I.vl[k] = reset(I.vl[k] + alpha_z * I.dvl[k], s + r);
      I.vu[k] = reset(I.vu[k] + alpha_z * I.dvu[k], r - s);
    }
  }
}

// Method constants: the augmented driver's (Waechter & Biegler 2006).
constexpr double MU_INIT = 0.1, KAPPA_MU = 0.2, THETA_MU = 1.5, KAPPA_EPS = 10.0;
constexpr double TAU_MIN = 0.99, S_MAX = 100.0, KAPPA_SIGMA = 1e10;
constexpr double GAMMA_THETA = 1e-5, GAMMA_PHI = 1e-5, DELTA = 1.0, S_THETA = 1.1, S_PHI = 2.3;
constexpr double ETA_PHI = 1e-4, GAMMA_ALPHA = 0.05;
constexpr double DW_MIN = 1e-20, DW_0 = 1e-4, DW_MAX = 1e40, KW_MINUS = 1.0 / 3.0, KW_PLUS = 8.0,
                 KW_PLUS_BAR = 100.0;
constexpr int REFINE_MAX = 20;
constexpr double REFINE_TOL = 1e-12;

}  // namespace

}  // namespace collo

using namespace collo;

extern "C" {

collo_status collo_lifted_ipm_solve(collo_problem* prob, const double* theta0, double relax,
                                    const collo_ipm_options* opts, collo_result* res) {
  if (!prob || !res || (prob->P.p > 0 && !theta0)) {
    set_error("NULL argument");
    return COLLO_ERR_INVALID_ARG;
  }
  if (!(relax > 0.0) || !std::isfinite(relax)) {
    set_error("relaxation must be finite and > 0");
    return COLLO_ERR_INVALID_ARG;
  }
  collo_ipm_options o;
  collo_ipm_options_default(&o);
  if (opts) o = *opts;
  COLLO_CUDA(cudaSetDevice(prob->device));
  const auto t_start = std::chrono::steady_clock::now();
  collo_status s = lifted_storage(prob);
  if (s != COLLO_OK) return s;
  LiftedStore& LS = *prob->lifted;
  DevLifted& L = LS.V;
  const DevProb& P = prob->P;
  const size_t nx = prob->n_x, nc = prob->n_c, nz = nx - P.p;
  const int p = P.p;
  cudaStream_t st = prob->stream;
  // device state (freed at return)
  DevArena mem;
  DevLiftedIpm I{};
  I.r = relax;
  I.s = mem.alloc<double>(nc); I.vl = mem.alloc<double>(nc); I.vu = mem.alloc<double>(nc);
  I.dvl = mem.alloc<double>(nc); I.dvu = mem.alloc<double>(nc); I.ss = mem.alloc<double>(nc);
  I.dzl = mem.alloc<double>(p); I.dzu = mem.alloc<double>(p); I.th = mem.alloc<double>(p);
  I.gneg = mem.alloc<double>(nx + nc);
  I.red = mem.alloc<double>(16);
  double* th0 = mem.alloc<double>(p);
  if (!I.s || !I.vl || !I.vu || !I.dvl || !I.dvu || !I.ss || !I.dzl || !I.dzu || !I.th ||
      !I.gneg || !I.red || !th0) {
    set_error("out of device memory for the lifted solve");
    return COLLO_ERR_OOM;
  }
  double* x = prob->x;
  double* lam = prob->lam;
  double* zl = prob->zl;
  double* zu = prob->zu;
  double* h = prob->hscal;   // pinned host mirror: h[56..63] for this driver
  auto fetch = [&](int first, int count) -> collo_status {
    COLLO_CUDA(cudaMemcpyAsync(h + 56, I.red + first, count * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
    COLLO_CUDA(cudaStreamSynchronize(st));
    return COLLO_OK;
  };
  // initial point: theta pushed, forward sweep, slacks c(x0) pushed into [-r, r]
  if (p) COLLO_CUDA(cudaMemcpyAsync(th0, theta0, p * sizeof(double), cudaMemcpyDefault, st));
  count_launch();
  k_lip_theta<<<1, 256, 0, st>>>(P, I, th0);
  COLLO_CUDA(cudaGetLastError());
  COLLO_CUDA(cudaStreamSynchronize(st));   // the sweep runs on the problem's runner stream
  int sweep_fail = 0;
  if ((s = collo_initial_states(prob, I.th, nullptr, &sweep_fail)) != COLLO_OK) return s;
  COLLO_CUDA(cudaMemsetAsync(lam, 0, nc * sizeof(double), st));
  COLLO_CUDA(launch_eval(P, prob->E, x, nullptr, 0.0, lam, 1.0, false, st));
  count_launch();
  k_lip_start<<<lifted_grid(nc), 256, 0, st>>>(P, prob->E, I, lam, zl, zu, nc);
  COLLO_CUDA(cudaGetLastError());

  double mu = MU_INIT, tau = std::max(TAU_MIN, 1.0 - mu);
  std::vector<std::pair<double, double>> filt;
  double dw_last = 0.0, theta_max = 0.0, theta_min = 0.0, err = INFINITY, phi = NAN;
  int acc = 0, it = 0, facs = 0, trials_all = 0, sweeps_all = 0;
  collo_status status = COLLO_ERR_MAXITER;
  const double m_pd = (double)nc, nb = 2.0 * p + 2.0 * nc;
  for (;;) {
    // evaluation with derivatives and the optimality measures
    COLLO_CUDA(launch_eval(P, prob->E, x, nullptr, 0.0, lam, 1.0, true, st));
    ++prob->eval_count;
    prob->evaluated = true;
    prob->factored = -1;
    COLLO_CUDA(launch_kkt_resid(P, prob->E, L.sigx, 0.0, 0.0, nullptr, lam, prob->E.grad, -1.0,
                                nullptr, 0.0, I.gneg, prob->thpart, prob->npart, nullptr,
                                prob->scal + 8, st));
    count_launch();
    k_lip_measures<<<1, IBS, 0, st>>>(P, prob->E, I, x, lam, zl, zu, nz, nc);
    COLLO_CUDA(cudaGetLastError());
    COLLO_CUDA(cudaMemcpyAsync(h + 52, prob->E.red, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                               st));
    if ((s = fetch(0, 8)) != COLLO_OK) return s;
    phi = h[52];
    if (!std::isfinite(phi) || !std::isfinite(h[53])) { status = COLLO_ERR_NUMERIC; break; }
    const double dmax = h[56], pmax = h[57], l1 = h[58], z1 = h[59], cmax = h[60],
                 cmin = h[61], theta_k = h[62], logs = h[63];
    if (it == 0) {
      theta_max = 1e4 * std::max(1.0, theta_k);
      theta_min = 1e-4 * std::max(1.0, theta_k);
    }
    const double s_d = std::max(S_MAX, (l1 + z1) / (m_pd + nb)) / S_MAX;
    const double s_c = std::max(S_MAX, z1 / nb) / S_MAX;
    auto E_mu = [&](double m) {
      const double compl_ = std::max(cmax - m, m - cmin);
      return std::max(std::max(dmax / s_d, pmax), compl_ / s_c);
    };
    err = E_mu(0.0);
    if (err <= o.tol) { status = COLLO_OK; break; }
    acc = err <= o.acceptable_tol ? acc + 1 : 0;
    if (acc >= o.acceptable_iter) { status = COLLO_ACCEPTABLE; break; }
    if (it >= o.max_iter) { status = COLLO_ERR_MAXITER; break; }
    const double wall =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (wall > o.max_wall_time) { status = COLLO_ERR_TIMEOUT; break; }
    while (E_mu(mu) <= KAPPA_EPS * mu) {
      const double nm = std::max(o.tol / 10.0, std::min(KAPPA_MU * mu, std::pow(mu, THETA_MU)));
      if (nm >= mu) break;
      mu = nm;
      tau = std::max(TAU_MIN, 1.0 - mu);
      filt.clear();
    }
    // right-hand sides and the lifted factorization with inertia correction
    count_launch();
    k_lip_rhs<<<lifted_grid(nx + nc), 256, 0, st>>>(P, prob->E, I, L, x, lam, zl, zu, mu, nz, nc);
    COLLO_CUDA(cudaGetLastError());
    double dw = 0.0;
    bool pd = false;
    ++facs;
    if ((s = lifted_factor_dev(prob, I.ss, 0.0, &pd)) != COLLO_OK) return s;
    if (!pd) {
      dw = dw_last == 0.0 ? DW_0 : std::max(DW_MIN, KW_MINUS * dw_last);
      for (;;) {
        ++facs;
        if ((s = lifted_factor_dev(prob, I.ss, dw, &pd)) != COLLO_OK) return s;
        if (pd) { dw_last = dw; break; }
        dw *= dw_last == 0.0 ? KW_PLUS_BAR : KW_PLUS;
        if (dw > DW_MAX) break;
      }
      if (!pd) { status = COLLO_ERR_INERTIA; break; }
    }
    int sw = 0;
    double rel = 0.0;
    if ((s = lifted_solve_dev(prob, REFINE_MAX, REFINE_TOL, &sw, &rel)) != COLLO_OK) {
      if (s == COLLO_ERR_NUMERIC) { status = s; break; }
      return s;
    }
    sweeps_all += sw;
    count_launch();
    k_lip_direction<<<1, IBS, 0, st>>>(P, prob->E, I, L, x, zl, zu, mu, tau, nz, nc);
    COLLO_CUDA(cudaGetLastError());
    if ((s = fetch(8, 3)) != COLLO_OK) return s;
    const double alpha_max = h[56], alpha_z = h[57], gphi = h[58];
    const double phi_k = phi - mu * logs;
    // backtracking filter line search (no second-order correction)
    double a_min;
    if (gphi < 0) {
      a_min = theta_k <= theta_min
                  ? GAMMA_ALPHA * std::min(GAMMA_THETA,
                                           std::min(GAMMA_PHI * theta_k / (-gphi),
                                                    DELTA * std::pow(theta_k, S_THETA) /
                                                        std::pow(-gphi, S_PHI)))
                  : GAMMA_ALPHA * std::min(GAMMA_THETA, GAMMA_PHI * theta_k / (-gphi));
    } else {
      a_min = GAMMA_ALPHA * GAMMA_THETA;
    }
    double alpha = alpha_max;
    bool accepted = false, ftype = false;
    while (alpha >= a_min) {
      ++trials_all;
      COLLO_CUDA(launch_eval(P, prob->E, x, L.dx, alpha, lam, 1.0, false, st));
      count_launch();
      k_lip_trial<<<1, IBS, 0, st>>>(P, prob->E, I, L, x, alpha, nz, nc);
      COLLO_CUDA(cudaGetLastError());
      COLLO_CUDA(cudaMemcpyAsync(h + 52, prob->E.red, sizeof(double), cudaMemcpyDeviceToHost, st));
      if ((s = fetch(11, 2)) != COLLO_OK) return s;
      const double phit = h[52], theta_t = h[56], phib_t = phit - mu * h[57];
      bool ok = false, ft = false;
      if (std::isfinite(theta_t) && std::isfinite(phib_t) && std::isfinite(phit) &&
          theta_t < theta_max) {
        bool in_filter = false;
        for (const auto& f : filt)
          if (theta_t >= f.first && phib_t >= f.second) { in_filter = true; break; }
        if (!in_filter) {
          const bool sw_ = gphi < 0 &&
                           alpha * std::pow(-gphi, S_PHI) > DELTA * std::pow(theta_k, S_THETA);
          if (theta_k <= theta_min && sw_) {
            ok = phib_t <= phi_k + ETA_PHI * alpha * gphi;
            ft = true;
          } else {
            ok = theta_t <= (1.0 - GAMMA_THETA) * theta_k || phib_t <= phi_k - GAMMA_PHI * theta_k;
          }
        }
      }
      if (ok) { accepted = true; ftype = ft; break; }
      alpha *= 0.5;
    }
    if (!accepted) { status = COLLO_ERR_LINESEARCH; break; }
    if (!ftype) filt.emplace_back((1.0 - GAMMA_THETA) * theta_k, phi_k - GAMMA_PHI * theta_k);
    count_launch();
    k_lip_update<<<lifted_grid(nx + nc), 256, 0, st>>>(P, I, L, x, lam, zl, zu, alpha, alpha_z, mu,
                                                       KAPPA_SIGMA, nz, nc);
    COLLO_CUDA(cudaGetLastError());
    if (o.verbose)
      std::printf("lifted it %d phi %.8e err %.3e mu %.2e dw %.2e alpha %.3e\n", it, phi, err, mu,
                  dw, alpha);
    ++it;
  }
  COLLO_CUDA(cudaStreamSynchronize(st));
  res->status = status;
  res->iterations = it;
  res->factorizations = facs;
  res->line_search_trials = trials_all;
  res->refinement_sweeps = sweeps_all;
  res->fp64_factorizations = facs;
  res->phi = phi;
  res->kkt_error = err;
  res->mu = mu;
  res->wall_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  if (res->theta && p)
    COLLO_CUDA(cudaMemcpyAsync(res->theta, x + nz, p * sizeof(double), cudaMemcpyDefault, st));
  if (res->x) COLLO_CUDA(cudaMemcpyAsync(res->x, x, nx * sizeof(double), cudaMemcpyDefault, st));
  if (res->lambda)
    COLLO_CUDA(cudaMemcpyAsync(res->lambda, lam, nc * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  return status;
}

}  // extern "C"
