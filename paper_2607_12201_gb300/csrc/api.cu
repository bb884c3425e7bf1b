// C ABI of libcollo: problem construction, evaluation, KKT factor / solve.
// The interior-point driver is in ipm.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <set>
#include <type_traits>

#include "problem.cuh"

namespace collo {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
static std::atomic<long long> g_launches{0};
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
Schedule& schedule() {
  static Schedule s;
  return s;
}

// Collocation tables (Eq. 2b, 2c).  Points: Radau IIA for K = 3, the
// roots of P_3 - P_2 on [0, 1] in closed form, tau = (4 -+ sqrt 6) / 10 and 1;
// Gauss-Legendre for K = 4, the roots of P_4 mapped from [-1, 1],
// x = +-sqrt(3/7 -+ (2/7) sqrt(6/5)), tau = (1 + x) / 2.  tau_0 = 0 in both.
// D[k][j] = l_j'(tau_k) from the barycentric weights
// w_j = 1 / prod_{l != j} (tau_j - tau_l):
//   D[k][j] = (w_j / w_k) / (tau_k - tau_j),  D[k][k] = -sum_{j != k} D[k][j];
// continuity weights b_j = l_j(1) (Radau: exactly delta_jK, as tau_K = 1).
static void colloc_tables(int gauss, double tau[NPMAX], double D[NPMAX][NPMAX],
                          double bw[NPMAX]) {
  const int np = gauss ? 5 : 4;
  tau[0] = 0.0;
  if (gauss) {
    const double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
    const double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
    tau[1] = 0.5 * (1.0 - b);
    tau[2] = 0.5 * (1.0 - a);
    tau[3] = 0.5 * (1.0 + a);
    tau[4] = 0.5 * (1.0 + b);
  } else {
    const double s6 = std::sqrt(6.0);
    tau[1] = (4.0 - s6) / 10.0;
    tau[2] = (4.0 + s6) / 10.0;
    tau[3] = 1.0;
  }
  double w[NPMAX];
  for (int j = 0; j < np; ++j) {
    w[j] = 1.0;
    for (int l = 0; l < np; ++l)
      if (l != j) w[j] /= (tau[j] - tau[l]);
  }
  for (int k = 0; k < np; ++k) {
    double sum = 0.0;
    for (int j = 0; j < np; ++j) {
      if (j == k) continue;
      D[k][j] = (w[j] / w[k]) / (tau[k] - tau[j]);
      sum += D[k][j];
    }
    D[k][k] = -sum;
  }
  for (int j = 0; j < np; ++j) {
    if (!gauss) { bw[j] = j == np - 1 ? 1.0 : 0.0; continue; }
    double v = 1.0;
    for (int l = 0; l < np; ++l)
      if (l != j) v *= (1.0 - tau[l]) / (tau[j] - tau[l]);
    bw[j] = v;
  }
  for (int j = np; j < NPMAX; ++j) {
    tau[j] = 0.0; bw[j] = 0.0;
    for (int k = 0; k < NPMAX; ++k) D[j][k] = D[k][j] = 0.0;
  }
}

// Every device array of a factorization store, in allocation order:
// fn(pointer member, element count).  Used both to allocate a store and to
// count its bytes before it exists (admission by memory budget).
template <typename T, class Fn>
static void factor_layout(const DevProb& P, int n_slabs, DevFactor<T>& F, Fn&& fn) {
  const size_t N = P.N, n = P.n, p = P.p;
  const size_t K = P.K;
  fn(F.Lel, N * 2 * K * n * P.ext);
  fn(F.Del, N * K * n * 3);
  fn(F.Aif, N * 4 * n * n);
  fn(F.Cpl, N * n * n);
  fn(F.Bif, N * 2 * n * p);
  fn(F.Lb, N * 2 * n * P.bext);
  fn(F.Db, N * n * 3);
  fn(F.Scon, 2 * N * p * p);
  fn(F.inert, 2 * N * 3);
  fn(F.Vint, N * 2 * K * n);
  fn(F.Rif, N * 2 * n);
  fn(F.Vb, N * 2 * n);
  fn(F.Rth, 2 * N * p);
  fn(F.chunkS, (size_t)CHUNKS * p * p);
  fn(F.chunkR, (size_t)CHUNKS * p);
  fn(F.gbar, (size_t)1);
  const size_t w = factor_work_elems<T>(P, n_slabs);
  if (w) fn(F.work, w);
}

template <typename T>
static int64_t factor_store_bytes(const collo_problem* pr) {
  DevFactor<T> F{};
  size_t b = 0;
  factor_layout<T>(pr->P, pr->n_slabs, F, [&](auto*& ptr, size_t cnt) {
    using U = std::remove_reference_t<decltype(*ptr)>;
    b += DevArena::bytes_of<U>(cnt);
  });
  return (int64_t)b;
}

template <typename T>
static collo_status alloc_factor(collo_problem* pr, FactorStore<T>& fs) {
  if (fs.allocated) return COLLO_OK;
  DevFactor<T>& F = fs.F;
  F = DevFactor<T>{};
  fs.mem.release(nullptr);
  fs.mem.stream = pr->stream;
  bool ok = true;
  factor_layout<T>(pr->P, pr->n_slabs, F, [&](auto*& ptr, size_t cnt) {
    using U = std::remove_reference_t<decltype(*ptr)>;
    ptr = fs.mem.template alloc<U>(cnt);
    ok = ok && ptr != nullptr;
  });
  if (!ok) {
    fs.mem.release(nullptr);
    F = DevFactor<T>{};
    set_error("device allocation failed for the factorization storage");
    return COLLO_ERR_OOM;
  }
  if (cudaMemsetAsync(F.gbar, 0, sizeof(GridBar), pr->stream) != cudaSuccess ||
      cudaStreamSynchronize(pr->stream) != cudaSuccess) {
    cudaGetLastError();
    set_error("initialising the factorization storage failed");
    return COLLO_ERR_DEVICE;
  }
  F.persistent = pr->launch_mode == 0 ? 1 : 0;
  F.n_slabs = pr->n_slabs;
  fs.allocated = true;
  return COLLO_OK;
}

template <typename T>
static void free_factor(FactorStore<T>& fs, cudaStream_t st) {
  fs.mem.release(st);
  fs.F = DevFactor<T>{};
  fs.allocated = false;
}

// Arrays of the second line-search trial and the spare Schur block (allocated
// once, with the first spare store): fn(pointer, count).
template <class Fn>
static void spare_eval_layout(collo_problem* pr, Fn&& fn) {
  const size_t p = pr->P.p;
  fn(pr->c_spare, (size_t)pr->n_c);
  fn(pr->part_spare, (size_t)pr->P.N * 4);
  fn(pr->red_spare, (size_t)8);
  DevSchur& S = pr->S_spare;
  fn(S.S, schur_doubles((int)p));
  fn(S.Sd, p);
  fn(S.xth, p);
  fn(S.inertia, (size_t)3);
  fn(S.diag, p);
}

collo_status ensure_factor_storage(collo_problem* pr, int precision) {
  return precision == COLLO_PRECISION_MIXED ? alloc_factor(pr, pr->f32) : alloc_factor(pr, pr->f64);
}

collo_status ensure_spare_storage(collo_problem* pr, int precision) {
  collo_status s = precision == COLLO_PRECISION_MIXED ? alloc_factor(pr, pr->f32_spare)
                                                       : alloc_factor(pr, pr->f64_spare);
  if (s != COLLO_OK || pr->spare_S) return s;
  DevArena& A = pr->arena;
  bool ok = true;
  spare_eval_layout(pr, [&](auto*& ptr, size_t cnt) {
    using U = std::remove_reference_t<decltype(*ptr)>;
    ptr = A.template alloc<U>(cnt);
    ok = ok && ptr != nullptr;
  });
  if (!ok) {
    set_error("device allocation failed for the spare evaluation / Schur storage");
    return COLLO_ERR_OOM;
  }
  pr->spare_S = true;
  return COLLO_OK;
}

int64_t problem_held_bytes(const collo_problem* pr) {
  return (int64_t)(pr->arena.bytes + pr->f64.mem.bytes + pr->f32.mem.bytes +
                   pr->f64_spare.mem.bytes + pr->f32_spare.mem.bytes);
}

int64_t problem_solve_bytes(const collo_problem* pr, int precision) {
  const bool mixed = precision == COLLO_PRECISION_MIXED;
  int64_t b = (int64_t)pr->arena.bytes;
  if (!pr->spare_S) {
    size_t e = 0;
    // the counting callback reads the sizes only; no pointer is written
    spare_eval_layout(const_cast<collo_problem*>(pr), [&](auto*& ptr, size_t cnt) {
      using U = std::remove_reference_t<decltype(*ptr)>;
      e += DevArena::bytes_of<U>(cnt);
    });
    b += (int64_t)e;
  }
  const int64_t s64 = factor_store_bytes<double>(pr), s32 = factor_store_bytes<float>(pr);
  // the FP64 store and its spare always; the FP32 pair for the mixed path
  b += pr->f64.allocated ? (int64_t)pr->f64.mem.bytes : s64;
  b += pr->f64_spare.allocated ? (int64_t)pr->f64_spare.mem.bytes : s64;
  if (mixed || pr->f32.allocated) b += pr->f32.allocated ? (int64_t)pr->f32.mem.bytes : s32;
  if (mixed || pr->f32_spare.allocated)
    b += pr->f32_spare.allocated ? (int64_t)pr->f32_spare.mem.bytes : s32;
  return b;
}

void release_factor_storage(collo_problem* pr, cudaStream_t st) {
  free_factor(pr->f64, st);
  free_factor(pr->f32, st);
  free_factor(pr->f64_spare, st);
  free_factor(pr->f32_spare, st);
  pr->factored = -1;
}

void swap_spare(collo_problem* pr, int precision) {
  if (precision == COLLO_PRECISION_MIXED) std::swap(pr->f32, pr->f32_spare);
  else std::swap(pr->f64, pr->f64_spare);
  std::swap(pr->S, pr->S_spare);
  pr->inst.S = pr->S;
}

static bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

}  // namespace collo

using namespace collo;

extern "C" {

const char* collo_last_error(void) { return g_last_error.c_str(); }
const char* collo_version(void) { return "collo 0.1 (sm_103a)"; }
long long collo_launch_count(void) { return g_launches.load(); }

collo_status collo_problem_create(const collo_network* net, const collo_observables* obs,
                                  const collo_data* data, const collo_mesh* mesh,
                                  const collo_problem_options* opts, collo_problem** out) {
  return collo_problem_create_conditions(net, obs, data, mesh, nullptr, opts, out);
}

collo_status collo_problem_create_conditions(const collo_network* net,
                                             const collo_observables* obs, const collo_data* data,
                                             const collo_mesh* mesh, const collo_conditions* conds,
                                             const collo_problem_options* opts,
                                             collo_problem** out) {
  if (!out) { set_error("out is NULL"); return COLLO_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!net || !mesh || !data || !obs) { set_error("NULL argument"); return COLLO_ERR_INVALID_ARG; }
  const int n = net->n_species, r = net->n_reactions, p = net->n_params;
  const int Nch = mesh->N, M = data->n_obs;
  const int Nc = conds ? conds->n_conditions : 1;
  if (n < 1 || r < 1 || p < 0 || Nch < 1 || M < 0 || Nc < 1) {
    set_error("bad sizes"); return COLLO_ERR_INVALID_ARG;
  }
  if ((long long)Nc * Nch > (1 << 30)) { set_error("too many elements"); return COLLO_ERR_INVALID_ARG; }
  const int N = Nc * Nch;   // elements of all conditions
  if (conds) {
    if (!conds->x0) { set_error("NULL condition initial states"); return COLLO_ERR_INVALID_ARG; }
    if (!finite_all(conds->x0, Nc * n)) {
      set_error("non-finite condition initial state"); return COLLO_ERR_INVALID_ARG;
    }
    if (conds->rate_scale)
      for (int k = 0; k < Nc * r; ++k)
        if (!std::isfinite(conds->rate_scale[k]) || !(conds->rate_scale[k] > 0)) {
          set_error("condition rate scales must be finite and > 0"); return COLLO_ERR_INVALID_ARG;
        }
    if (conds->obs_condition)
      for (int m = 0; m < M; ++m)
        if (conds->obs_condition[m] < 0 || conds->obs_condition[m] >= Nc) {
          set_error("bad measurement condition"); return COLLO_ERR_INVALID_ARG;
        }
  }
  if (mesh->scheme != COLLO_SCHEME_RADAU && mesh->scheme != COLLO_SCHEME_GAUSS) {
    set_error("unknown collocation scheme"); return COLLO_ERR_INVALID_ARG;
  }
  const int gauss = mesh->scheme == COLLO_SCHEME_GAUSS ? 1 : 0;
  if (mesh->K != (gauss ? 4 : 3)) {
    set_error("K must be 3 with Radau IIA points and 4 with Gauss-Legendre points");
    return COLLO_ERR_INVALID_ARG;
  }
  if (!(mesh->T > 0) || !std::isfinite(mesh->T)) { set_error("T must be positive"); return COLLO_ERR_INVALID_ARG; }
  if (!net->reactants || !net->products || !net->param_index || !net->k_fixed ||
      (!conds && !net->x0) ||
      (p > 0 && (!net->theta_lo || !net->theta_hi))) {
    set_error("NULL network array"); return COLLO_ERR_INVALID_ARG;
  }
  if (M > 0 && (!data->t || !data->observable || !data->y || !data->sigma || !obs->species)) {
    set_error("NULL data array"); return COLLO_ERR_INVALID_ARG;
  }
  for (int j = 0; j < r; ++j) {
    int a = net->reactants[2 * j], b = net->reactants[2 * j + 1];
    if (a < 0 || a >= n || b < -1 || b >= n) { set_error("bad reactant index"); return COLLO_ERR_INVALID_ARG; }
    for (int k = 0; k < 2; ++k) {
      int s = net->products[2 * j + k];
      if (s < -1 || s >= n) { set_error("bad product index"); return COLLO_ERR_INVALID_ARG; }
    }
    int q = net->param_index[j];
    if (q < -1 || q >= p) { set_error("bad parameter index"); return COLLO_ERR_INVALID_ARG; }
    if (q < 0 && !std::isfinite(net->k_fixed[j])) { set_error("non-finite fixed rate"); return COLLO_ERR_INVALID_ARG; }
  }
  if (!conds && !finite_all(net->x0, n)) { set_error("non-finite x0"); return COLLO_ERR_INVALID_ARG; }
  for (int q = 0; q < p; ++q)
    if (!std::isfinite(net->theta_lo[q]) || !std::isfinite(net->theta_hi[q]) ||
        !(net->theta_lo[q] < net->theta_hi[q])) {
      set_error("parameter bounds must be finite with lo < hi"); return COLLO_ERR_INVALID_ARG;
    }
  for (int m = 0; m < M; ++m) {
    int o = data->observable[m];
    if (o < 0 || o >= obs->n_observables) { set_error("bad observable index"); return COLLO_ERR_INVALID_ARG; }
    int s = obs->species[o];
    if (s < 0 || s >= n) { set_error("bad observed species"); return COLLO_ERR_INVALID_ARG; }
    if (!std::isfinite(data->t[m]) || !std::isfinite(data->y[m]) || !(data->sigma[m] > 0) ||
        !std::isfinite(data->sigma[m]) || data->t[m] < 0 || data->t[m] > mesh->T) {
      set_error("bad measurement (non-finite, sigma <= 0 or t outside [0, T])");
      return COLLO_ERR_INVALID_ARG;
    }
  }
  int dev = opts ? opts->device : 0;
  if (cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaSetDevice failed (no CUDA device?)");
    return COLLO_ERR_DEVICE;
  }
  std::unique_ptr<collo_problem> pr(new collo_problem());
  pr->device = dev;
  {
    HostInputs& h = pr->host;
    h.react.assign(net->reactants, net->reactants + 2 * r);
    h.prod.assign(net->products, net->products + 2 * r);
    h.pidx.assign(net->param_index, net->param_index + r);
    h.kfix.assign(net->k_fixed, net->k_fixed + r);
    if (conds) h.cond_x0.assign(conds->x0, conds->x0 + (size_t)Nc * n);
    else h.cond_x0.assign(net->x0, net->x0 + n);
    h.x0 = std::vector<double>(h.cond_x0.begin(), h.cond_x0.begin() + n);
    h.n_conditions = Nc;
    if (conds && conds->rate_scale)
      h.cond_scale.assign(conds->rate_scale, conds->rate_scale + (size_t)Nc * r);
    if (conds && conds->obs_condition && M > 0)
      h.obs_cond.assign(conds->obs_condition, conds->obs_condition + M);
    if (p > 0) {
      h.lo.assign(net->theta_lo, net->theta_lo + p);
      h.hi.assign(net->theta_hi, net->theta_hi + p);
    }
    if (M > 0) {
      h.species.assign(obs->species, obs->species + obs->n_observables);
      h.t.assign(data->t, data->t + M);
      h.observable.assign(data->observable, data->observable + M);
      h.y.assign(data->y, data->y + M);
      h.sigma.assign(data->sigma, data->sigma + M);
    }
  }
  pr->precision = opts ? opts->precision : 0;
  pr->launch_mode = opts ? opts->launch_mode : 0;
  if (pr->launch_mode != 0 && pr->launch_mode != 1) {
    set_error("launch_mode must be 0 or 1");
    return COLLO_ERR_INVALID_ARG;
  }
  if (opts && opts->stream) {
    pr->stream = (cudaStream_t)opts->stream;
  } else {
    COLLO_CUDA(cudaStreamCreateWithFlags(&pr->stream, cudaStreamNonBlocking));
    pr->own_stream = true;
  }
  DevProb& P = pr->P;
  P.n = n; P.r = r; P.p = p; P.N = N; P.M = M;
  P.Nc = Nc; P.Nch = Nch;
  P.K = mesh->K; P.np = P.K + 1; P.gauss = gauss; P.cpt = gauss ? 0 : P.K;
  P.m = 2 * P.np * n; P.ext = P.m + p; P.bext = 4 * n + p;
  P.logscale = net->log10_params ? 1 : 0;
  P.T = mesh->T; P.h = mesh->T / Nch;
  colloc_tables(gauss, P.tau, P.D, P.bw);
  pr->n_x = (int64_t)n * N * P.np + p;
  pr->n_c = (int64_t)n * N * P.np;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // global slabs of the blocks too large for shared memory: one per CUDA block
  // that may run at once, two per SM; not limited by N, since a batch's
  // kernels take their grid from the smallest slab count of its members
  pr->n_slabs = 2 * std::max(1, sms);

  // host-side CSR structures (index bookkeeping only)
  std::vector<int> nu_ptr(n + 1, 0), nu_r, rs_ptr(n + 1, 0), rs_r, pr_ptr(p + 1, 0), pr_r;
  std::vector<double> nu_v;
  {
    std::vector<std::vector<std::pair<int, double>>> lists(n);
    std::vector<std::vector<int>> cons(n);
    std::vector<std::vector<int>> pl(p);
    for (int j = 0; j < r; ++j) {
      std::vector<double> nu(n, 0.0);
      for (int k = 0; k < 2; ++k) {
        int a = net->reactants[2 * j + k];
        if (a >= 0) nu[a] -= 1.0;
        int b = net->products[2 * j + k];
        if (b >= 0) nu[b] += 1.0;
      }
      for (int s = 0; s < n; ++s)
        if (nu[s] != 0.0) lists[s].push_back({j, nu[s]});
      int a = net->reactants[2 * j], b = net->reactants[2 * j + 1];
      cons[a].push_back(j);
      if (b >= 0 && b != a) cons[b].push_back(j);
      if (net->param_index[j] >= 0) pl[net->param_index[j]].push_back(j);
    }
    for (int s = 0; s < n; ++s) {
      nu_ptr[s + 1] = nu_ptr[s] + (int)lists[s].size();
      for (auto& e : lists[s]) { nu_r.push_back(e.first); nu_v.push_back(e.second); }
      rs_ptr[s + 1] = rs_ptr[s] + (int)cons[s].size();
      for (int j : cons[s]) rs_r.push_back(j);
    }
    for (int q = 0; q < p; ++q) {
      pr_ptr[q + 1] = pr_ptr[q] + (int)pl[q].size();
      for (int j : pl[q]) pr_r.push_back(j);
    }
  }
  // structural nonzeros of the derivative blocks (the eval kernels accumulate
  // JZ / JT over the reactions changing a species, Wzz / Wzt over the
  // reactions consuming it): sorted index sets per row or column
  std::vector<std::set<int>> jzr(n), jzc(n), wzr(n), wtr(n), jtr(n), thq(p);
  for (int j = 0; j < r; ++j) {
    const int a = net->reactants[2 * j], b = net->reactants[2 * j + 1];
    const int q = net->param_index[j];
    std::vector<double> nu(n, 0.0);
    for (int k = 0; k < 2; ++k) {
      if (net->reactants[2 * j + k] >= 0) nu[net->reactants[2 * j + k]] -= 1.0;
      if (net->products[2 * j + k] >= 0) nu[net->products[2 * j + k]] += 1.0;
    }
    for (int s2 = 0; s2 < n; ++s2) {
      if (nu[s2] == 0.0) continue;
      jzr[s2].insert(a);
      if (b >= 0) jzr[s2].insert(b);
      if (q >= 0) { jtr[s2].insert(q); thq[q].insert(s2); }
    }
    if (b >= 0) {
      if (a == b) wzr[a].insert(a);
      else { wzr[a].insert(b); wzr[b].insert(a); }
    }
    if (q >= 0) {
      wtr[a].insert(q); thq[q].insert(a);
      if (b >= 0) { wtr[b].insert(q); thq[q].insert(b); }
    }
  }
  for (int s2 = 0; s2 < n; ++s2)
    for (int t : jzr[s2]) jzc[t].insert(s2);
  // observations: element from the same rule the kernels use, grouped by element
  std::vector<int> oelem(M);
  for (int m = 0; m < M; ++m) {
    double u = data->t[m] * Nch / mesh->T;
    int i = (int)std::ceil(u) - 1;
    const int c = (conds && conds->obs_condition) ? conds->obs_condition[m] : 0;
    oelem[m] = c * Nch + std::min(std::max(i, 0), Nch - 1);
  }
  std::vector<int> order(M);
  for (int m = 0; m < M; ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return oelem[a] < oelem[b]; });
  std::vector<int> obs_ptr(N + 1, 0), obs_s(M);
  std::vector<double> obs_t(M), obs_y(M), obs_sig(M);
  for (int k = 0; k < M; ++k) {
    int m = order[k];
    obs_ptr[oelem[m] + 1]++;
    obs_s[k] = obs->species[data->observable[m]];
    obs_t[k] = data->t[m];
    obs_y[k] = data->y[m];
    obs_sig[k] = data->sigma[m];
  }
  for (int i = 0; i < N; ++i) obs_ptr[i + 1] += obs_ptr[i];

  DevArena& A = pr->arena;
  auto up_i = [&](const int* h, size_t cnt) -> const int* {
    int* d = A.alloc<int>(cnt);
    if (d && cnt) cudaMemcpy(d, h, cnt * sizeof(int), cudaMemcpyDefault);
    return d;
  };
  auto up_d = [&](const double* h, size_t cnt) -> const double* {
    double* d = A.alloc<double>(cnt);
    if (d && cnt) cudaMemcpy(d, h, cnt * sizeof(double), cudaMemcpyDefault);
    return d;
  };
  P.react = up_i(net->reactants, 2 * (size_t)r);
  P.prod = up_i(net->products, 2 * (size_t)r);
  P.pidx = up_i(net->param_index, r);
  P.kfix = up_d(net->k_fixed, r);
  P.x0 = up_d(pr->host.cond_x0.data(), (size_t)Nc * n);
  P.kscale = pr->host.cond_scale.empty() ? nullptr
                                          : up_d(pr->host.cond_scale.data(), (size_t)Nc * r);
  P.theta_lo = up_d(p ? net->theta_lo : nullptr, p);
  P.theta_hi = up_d(p ? net->theta_hi : nullptr, p);
  P.nu_ptr = up_i(nu_ptr.data(), n + 1);
  P.nu_r = up_i(nu_r.data(), nu_r.size());
  P.nu_v = up_d(nu_v.data(), nu_v.size());
  P.rs_ptr = up_i(rs_ptr.data(), n + 1);
  P.rs_r = up_i(rs_r.data(), rs_r.size());
  P.pr_ptr = up_i(pr_ptr.data(), p + 1);
  P.pr_r = up_i(pr_r.data(), pr_r.size());
  bool pat_ok = true;
  auto up_csr = [&](const std::vector<std::set<int>>& sets, const int*& ptr, const int*& idx) {
    std::vector<int> hp(sets.size() + 1, 0), hi;
    for (size_t k = 0; k < sets.size(); ++k) {
      hi.insert(hi.end(), sets[k].begin(), sets[k].end());
      hp[k + 1] = (int)hi.size();
    }
    if (hi.empty()) hi.push_back(0);   // never read: every row range is empty
    ptr = up_i(hp.data(), hp.size());
    idx = up_i(hi.data(), hi.size());
    pat_ok = pat_ok && ptr && idx;
  };
  up_csr(jzr, P.jzr_ptr, P.jzr_i);
  up_csr(jzc, P.jzc_ptr, P.jzc_i);
  up_csr(wzr, P.wzr_ptr, P.wzr_i);
  up_csr(wtr, P.wtr_ptr, P.wtr_i);
  up_csr(jtr, P.jtr_ptr, P.jtr_i);
  up_csr(thq, P.thq_ptr, P.thq_i);
  {
    std::vector<int> osp(n, 0);
    for (int k = 0; k < M; ++k) osp[obs_s[k]] = 1;
    P.obs_sp = up_i(osp.data(), n);
    pat_ok = pat_ok && P.obs_sp;
  }
  P.obs_ptr = up_i(obs_ptr.data(), N + 1);
  P.obs_s = up_i(obs_s.data(), M);
  P.obs_y = up_d(obs_y.data(), M);
  P.obs_sig = up_d(obs_sig.data(), M);
  const double* d_obs_t = up_d(obs_t.data(), M);
  double* obs_w = A.alloc<double>((size_t)M * P.np);
  int* obs_elem_chk = A.alloc<int>(M);
  P.obs_w = obs_w;
  const size_t NN = (size_t)N, nn = (size_t)n * n, np_ = (size_t)n * p;
  DevEval& E = pr->E;
  E.c = A.alloc<double>(pr->n_c);
  E.grad = A.alloc<double>(pr->n_x);
  E.JZ = A.alloc<double>(NN * P.K * nn);
  E.JT = A.alloc<double>(NN * P.K * np_);
  E.Wzz = A.alloc<double>(NN * P.K * nn);
  E.Wzt = A.alloc<double>(NN * P.K * np_);
  E.Wobj = A.alloc<double>(NN * n * P.np * P.np);
  E.part = A.alloc<double>(NN * 4);
  E.wtt_part = A.alloc<double>(NN * p);
  E.red = A.alloc<double>(8);
  E.wtt = A.alloc<double>(p);
  DevSchur& S = pr->S;
  S.S = A.alloc<double>(schur_doubles(p));
  S.Sd = A.alloc<double>(p);
  S.xth = A.alloc<double>(p);
  S.inertia = A.alloc<long long>(3);
  S.diag = A.alloc<double>(p);
  const size_t nk = pr->n_x + pr->n_c;
  pr->sigma = A.alloc<double>(pr->n_x);
  pr->kvec_a = A.alloc<double>(nk);
  pr->kvec_b = A.alloc<double>(nk);
  pr->kvec_r = A.alloc<double>(nk);
  pr->kvec_c = A.alloc<double>(nk);
  pr->thpart = A.alloc<double>(NN * p + (size_t)CHUNKS * p);
  pr->npart = A.alloc<double>(NN * 3);
  pr->scal = A.alloc<double>(64);
  pr->red_parts = A.alloc<double>(256);
  pr->x = A.alloc<double>(pr->n_x);
  pr->lam = A.alloc<double>(pr->n_c);
  pr->zl = A.alloc<double>(p);
  pr->zu = A.alloc<double>(p);
  pr->dz = A.alloc<double>(2 * (size_t)p);
  pr->thx = A.alloc<double>(8 * (size_t)p + 8);
  pr->fails = A.alloc<int>(1);
  const size_t sweep_dim = (size_t)P.K * n;
  const bool sweep_global = sweep_dim * (sweep_dim + 1) * sizeof(float) > 160 * 1024;
  if (sweep_global) pr->sweep_work = A.alloc<float>(sweep_dim * (sweep_dim + 1));
  bool ok = P.react && P.prod && P.pidx && P.kfix && P.x0 && P.theta_lo && P.theta_hi &&
            (pr->host.cond_scale.empty() || P.kscale) &&
            P.nu_ptr && P.nu_r && P.nu_v && P.rs_ptr && P.rs_r && P.pr_ptr && P.pr_r && pat_ok &&
            P.obs_ptr && P.obs_s && P.obs_y && P.obs_sig && d_obs_t && obs_w && obs_elem_chk &&
            E.c && E.grad && E.JZ && E.JT && E.Wzz && E.Wzt && E.Wobj && E.part && E.wtt_part &&
            E.red && E.wtt && S.S && S.Sd && S.xth && S.inertia && S.diag && pr->sigma &&
            pr->kvec_a && pr->kvec_b && pr->kvec_r && pr->kvec_c && pr->thpart && pr->npart &&
            pr->scal && pr->red_parts && pr->x && pr->lam && pr->zl && pr->zu && pr->dz && pr->thx && pr->fails &&
            (!sweep_global || pr->sweep_work);
  if (!ok) { set_error("device allocation failed"); return COLLO_ERR_OOM; }
  if (cudaMallocHost(&pr->hscal, 64 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    set_error("pinned host allocation failed");
    return COLLO_ERR_OOM;
  }
  {
    DevInst& I = pr->inst;
    I.P = P; I.E = E; I.S = S;
    I.sigma = pr->sigma; I.x = pr->x; I.lam = pr->lam; I.zl = pr->zl; I.zu = pr->zu;
    I.dz = pr->dz; I.bar = pr->thx; I.zlmzu = pr->thx + p; I.th0 = pr->thx + 2 * (size_t)p;
    I.ka = pr->kvec_a; I.kb = pr->kvec_b; I.kr = pr->kvec_r; I.kc = pr->kvec_c;
    I.thpart = pr->thpart; I.npart = pr->npart; I.fails = pr->fails; I.sweep_work = pr->sweep_work;
    I.n_x = pr->n_x; I.n_c = pr->n_c;
  }
  COLLO_CUDA(cudaMemsetAsync(pr->sigma, 0, pr->n_x * sizeof(double), pr->stream));
  COLLO_CUDA(launch_obs_weights(P, M, Nch, mesh->T, d_obs_t, obs_elem_chk, obs_w, pr->stream));
  COLLO_CUDA(cudaStreamSynchronize(pr->stream));
  COLLO_CUDA(cudaGetLastError());
  *out = pr.release();
  return COLLO_OK;
}

void collo_problem_destroy(collo_problem* prob) {
  if (!prob) return;
  cudaSetDevice(prob->device);
  cudaStreamSynchronize(prob->stream);
  if (prob->hscal) cudaFreeHost(prob->hscal);
  if (prob->own_stream) cudaStreamDestroy(prob->stream);
  delete prob;
}

collo_status collo_problem_sizes(const collo_problem* prob, collo_sizes* out) {
  if (!prob || !out) { set_error("NULL argument"); return COLLO_ERR_INVALID_ARG; }
  out->n = prob->P.n; out->r = prob->P.r; out->p = prob->P.p; out->N = prob->P.N;
  out->K = prob->P.K; out->M = prob->P.M; out->n_x = prob->n_x; out->n_c = prob->n_c;
  out->levels = bcr_levels(prob->P.N);
  out->device_bytes = problem_held_bytes(prob);
  out->n_conditions = prob->P.Nc;
  out->elements_per_condition = prob->P.Nch;
  return COLLO_OK;
}

void* collo_problem_stream(const collo_problem* prob) { return prob ? (void*)prob->stream : nullptr; }

collo_status collo_problem_solve_bytes(const collo_problem* prob, int precision, int64_t* bytes) {
  if (!prob || !bytes) { set_error("NULL argument"); return COLLO_ERR_INVALID_ARG; }
  if (precision != COLLO_PRECISION_FP64 && precision != COLLO_PRECISION_MIXED) {
    set_error("bad precision"); return COLLO_ERR_INVALID_ARG;
  }
  *bytes = problem_solve_bytes(prob, precision);
  return COLLO_OK;
}

collo_status collo_eval(collo_problem* prob, const double* x, const double* lambda,
                        double obj_factor, collo_eval_out* out) {
  if (!prob || !x) { set_error("NULL argument"); return COLLO_ERR_INVALID_ARG; }
  COLLO_CUDA(cudaSetDevice(prob->device));
  cudaStream_t st = prob->stream;
  const DevProb& P = prob->P;
  const DevEval& E = prob->E;
  double* dx = prob->kvec_c;                    // staging for x
  double* dl = prob->kvec_c + prob->n_x;       // staging for lambda
  COLLO_CUDA(cudaMemcpyAsync(dx, x, prob->n_x * sizeof(double), cudaMemcpyDefault, st));
  if (lambda)
    COLLO_CUDA(cudaMemcpyAsync(dl, lambda, prob->n_c * sizeof(double), cudaMemcpyDefault, st));
  else
    COLLO_CUDA(cudaMemsetAsync(dl, 0, prob->n_c * sizeof(double), st));
  if (prob->launch_mode == 0) {
    collo_status s = runner_eval(prob, obj_factor);
    if (s != COLLO_OK) return s;
  } else {
    COLLO_CUDA(launch_eval(P, E, dx, nullptr, 0.0, dl, obj_factor, true, st));
  }
  const size_t NN = P.N, nn = (size_t)P.n * P.n, np_ = (size_t)P.n * P.p;
  if (out) {
    auto cp = [&](double* dst, const double* src, size_t cnt) -> cudaError_t {
      if (!dst || cnt == 0) return cudaSuccess;
      return cudaMemcpyAsync(dst, src, cnt * sizeof(double), cudaMemcpyDefault, st);
    };
    COLLO_CUDA(cp(out->phi, E.red, 1));
    COLLO_CUDA(cp(out->c, E.c, prob->n_c));
    COLLO_CUDA(cp(out->grad, E.grad, prob->n_x));
    COLLO_CUDA(cp(out->jac_z, E.JZ, NN * P.K * nn));
    COLLO_CUDA(cp(out->jac_theta, E.JT, NN * P.K * np_));
    COLLO_CUDA(cp(out->hess_zz, E.Wzz, NN * P.K * nn));
    COLLO_CUDA(cp(out->hess_ztheta, E.Wzt, NN * P.K * np_));
    COLLO_CUDA(cp(out->hess_thth, E.wtt, P.p));
    COLLO_CUDA(cp(out->hess_obj, E.Wobj, NN * P.n * P.np * P.np));
  }
  COLLO_CUDA(cudaMemcpyAsync(prob->hscal, E.red, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  prob->evaluated = true;
  ++prob->eval_count;
  prob->factored = -1;
  if (!std::isfinite(prob->hscal[0]) || !std::isfinite(prob->hscal[1])) {
    set_error("non-finite objective or constraint values");
    return COLLO_ERR_NUMERIC;
  }
  return COLLO_OK;
}

}  // extern "C"

namespace collo {

// Factor with the sigma already in prob->sigma; reads back the inertia.
collo_status factor_internal(collo_problem* prob, double dw, double dc, int precision,
                             long long inertia[3]) {
  collo_status s = ensure_factor_storage(prob, precision);
  if (s != COLLO_OK) return s;
  cudaStream_t st = prob->stream;
  if (precision == COLLO_PRECISION_MIXED)
    COLLO_CUDA(launch_factor<float>(prob->P, prob->E, prob->sigma, dw, dc, prob->f32.F, prob->S, st));
  else
    COLLO_CUDA(launch_factor<double>(prob->P, prob->E, prob->sigma, dw, dc, prob->f64.F, prob->S, st));
  COLLO_CUDA(cudaMemcpyAsync(prob->hscal + 40, prob->S.inertia, 3 * sizeof(long long),
                             cudaMemcpyDeviceToHost, st));
  GridBar* gb = precision == COLLO_PRECISION_MIXED ? prob->f32.F.gbar : prob->f64.F.gbar;
  COLLO_CUDA(cudaMemcpyAsync(prob->hscal + 44, &gb->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  std::memcpy(inertia, prob->hscal + 40, 3 * sizeof(long long));
  int berr = 0;
  std::memcpy(&berr, prob->hscal + 44, sizeof(int));
  if (berr) {
    cudaMemsetAsync(&gb->err, 0, sizeof(int), st);
    set_error("grid barrier of the factorization kernel timed out");
    return COLLO_ERR_TIMEOUT;
  }
  prob->factored = precision;
  prob->fac_dw = dw;
  prob->fac_dc = dc;
  return COLLO_OK;
}

// Solve K sol = b (device vectors, may not alias) with FP64 iterative refinement.
collo_status solve_internal(collo_problem* prob, const double* b, double* sol, int refine_max,
                            double refine_tol, int* sweeps, double* resid) {
  cudaStream_t st = prob->stream;
  const DevProb& P = prob->P;
  const size_t nk = prob->n_x + prob->n_c;
  auto inner = [&](const double* rhs, double* out) -> cudaError_t {
    if (prob->factored == COLLO_PRECISION_MIXED)
      return launch_solve<float>(P, prob->f32.F, prob->S, rhs, out, st);
    return launch_solve<double>(P, prob->f64.F, prob->S, rhs, out, st);
  };
  COLLO_CUDA(inner(b, sol));
  int k = 0;
  double rel = 0.0;
  for (;;) {
    COLLO_CUDA(launch_kkt_resid(P, prob->E, prob->sigma, prob->fac_dw, prob->fac_dc, sol,
                                sol + prob->n_x, b, 1.0, b + prob->n_x, 1.0, prob->kvec_r,
                                prob->thpart, prob->npart, nullptr, prob->scal + 8, st));
    COLLO_CUDA(cudaMemcpyAsync(prob->hscal + 8, prob->scal + 8, 3 * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
    GridBar* gb = prob->factored == COLLO_PRECISION_MIXED ? prob->f32.F.gbar : prob->f64.F.gbar;
    COLLO_CUDA(cudaMemcpyAsync(prob->hscal + 12, &gb->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    COLLO_CUDA(cudaStreamSynchronize(st));
    int berr = 0;
    std::memcpy(&berr, prob->hscal + 12, sizeof(int));
    if (berr) {
      cudaMemsetAsync(&gb->err, 0, sizeof(int), st);
      set_error("grid barrier of the solve kernel timed out");
      return COLLO_ERR_TIMEOUT;
    }
    double rn = std::max(prob->hscal[8], prob->hscal[9]);
    double bn = std::max(1.0, prob->hscal[10]);
    rel = rn / bn;
    if (!(rel > refine_tol) || k >= refine_max || !std::isfinite(rel)) break;
    COLLO_CUDA(inner(prob->kvec_r, prob->kvec_c));
    ++k;
    COLLO_CUDA(launch_axpy(sol, prob->kvec_c, 1.0, nk, st));   // sol += correction
  }
  if (sweeps) *sweeps = k;
  if (resid) *resid = rel;
  if (!std::isfinite(rel)) { set_error("non-finite KKT solution"); return COLLO_ERR_NUMERIC; }
  return COLLO_OK;
}

}  // namespace collo

extern "C" {

collo_status collo_kkt_factor(collo_problem* prob, const double* sigma, double delta_w,
                              double delta_c, int precision, collo_inertia* out) {
  if (!prob) { set_error("NULL problem"); return COLLO_ERR_INVALID_ARG; }
  if (!prob->evaluated) { set_error("collo_eval has not run"); return COLLO_ERR_NOT_EVALUATED; }
  if (!std::isfinite(delta_w) || !std::isfinite(delta_c) || delta_w < 0 || delta_c < 0) {
    set_error("regularisation must be finite and >= 0"); return COLLO_ERR_INVALID_ARG;
  }
  COLLO_CUDA(cudaSetDevice(prob->device));
  if (precision < 0) precision = prob->precision;
  if (precision != COLLO_PRECISION_FP64 && precision != COLLO_PRECISION_MIXED) {
    set_error("bad precision"); return COLLO_ERR_INVALID_ARG;
  }
  if (sigma)
    COLLO_CUDA(cudaMemcpyAsync(prob->sigma, sigma, prob->n_x * sizeof(double), cudaMemcpyDefault,
                               prob->stream));
  else
    COLLO_CUDA(cudaMemsetAsync(prob->sigma, 0, prob->n_x * sizeof(double), prob->stream));
  long long in[3];
  collo_status s = prob->launch_mode == 0 ? runner_factor(prob, precision, delta_w, delta_c, in)
                                          : factor_internal(prob, delta_w, delta_c, precision, in);
  if (s != COLLO_OK) return s;
  if (out) { out->n_pos = in[0]; out->n_neg = in[1]; out->n_zero = in[2]; }
  return COLLO_OK;
}

collo_status collo_kkt_solve(collo_problem* prob, const double* rhs, double* sol, int refine_max,
                             double refine_tol, collo_solve_info* info) {
  if (!prob || !rhs || !sol) { set_error("NULL argument"); return COLLO_ERR_INVALID_ARG; }
  if (prob->factored < 0) { set_error("no factorization"); return COLLO_ERR_NOT_FACTORED; }
  COLLO_CUDA(cudaSetDevice(prob->device));
  const size_t nk = prob->n_x + prob->n_c;
  cudaStream_t st = prob->stream;
  COLLO_CUDA(cudaMemcpyAsync(prob->kvec_a, rhs, nk * sizeof(double), cudaMemcpyDefault, st));
  int sweeps = 0;
  double resid = 0.0;
  collo_status s =
      prob->launch_mode == 0
          ? runner_solve(prob, refine_max < 0 ? 0 : refine_max, refine_tol, &sweeps, &resid)
          : solve_internal(prob, prob->kvec_a, prob->kvec_b, refine_max < 0 ? 0 : refine_max,
                           refine_tol, &sweeps, &resid);
  if (s != COLLO_OK) return s;
  COLLO_CUDA(cudaMemcpyAsync(sol, prob->kvec_b, nk * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  if (info) { info->refinement_sweeps = sweeps; info->residual = resid; }
  return COLLO_OK;
}

}  // extern "C"
