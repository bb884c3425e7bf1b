// Mesh refinement on the GPU: the collocation defect of a solution, its
// interpolation onto a finer mesh, warm starts, and a batched
// refine-and-resolve loop.
//
// The paper observes that a collocation mesh fixed at the nominal parameters
// may be too coarse for the stiff dynamics near the optimum, and names
// adaptive refinement of the interval width as the remedy, usually run
// sequentially in an outer loop (Section "Static collocation mesh
// limitations"; Conclusion).  Here the outer loop is batched: every problem
// whose solve converged with a defect above the tolerance is re-created on a
// mesh of twice as many elements, warm-started from its interpolated
// solution, and all of them are solved again together in one batch.
//
// Defect of element i: the collocation polynomial z_i(tau) = sum_j l_j(tau)
// z_ij satisfies the ODE exactly at the K collocation points; at the
// midpoints tau*_m = (tau_(m-1) + tau_m) / 2, m = 1..K, between consecutive
// interpolation points it leaves the residual
//   d_ims = sum_j l_j'(tau*_m) z_ijs - h f_s(z_i(tau*_m), theta)
// (h times the residual of dz/dt = f), and the element's defect is
// max_{m,s} |d_ims|, an estimate of the local error in state units.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "problem.cuh"

namespace collo {

constexpr int DEF_BS = 128;

// Lagrange basis on the interpolation points tau[0..K]: l_j(t) and l_j'(t).
__device__ inline void lagrange(const DevProb& P, double t, double* l, double* dl) {
  for (int j = 0; j < P.np; ++j) {
    double v = 1.0, d = 0.0;
    for (int a = 0; a < P.np; ++a) {
      if (a == j) continue;
      const double inv = 1.0 / (P.tau[j] - P.tau[a]);
      // product rule: d/dt prod (t - tau_a) inv
      d = d * (t - P.tau[a]) * inv + v * inv;
      v *= (t - P.tau[a]) * inv;
    }
    l[j] = v;
    if (dl) dl[j] = d;
  }
}

// One block per element: the defect d_i (above) into def[i].
__global__ void __launch_bounds__(DEF_BS)
k_defect(DevProb P, const double* __restrict__ x, double* __restrict__ def) {
  extern __shared__ double sm[];
  const int n = P.n, r = P.r, i = blockIdx.x, tid = threadIdx.x;
  const int K = P.K, np = P.np;
  double* ze = sm;                 // [K+1][n] element states
  double* zt = ze + np * n;        // [K][n] z(tau*_m)
  double* dz = zt + K * n;         // [K][n] sum_j l_j'(tau*_m) z_j
  double* kr = dz + K * n;         // [r] rate constants
  double* mon = kr + r;            // [K][r] k_r prod of reactants at tau*_m
  __shared__ double red[DEF_BS];
  const size_t zoff = (size_t)i * np * n, nz = (size_t)P.N * np * n;
  for (int t = tid; t < np * n; t += DEF_BS) ze[t] = x[zoff + t];
  for (int j = tid; j < r; j += DEF_BS) {
    const int q = P.pidx[j];
    double k = q < 0 ? P.kfix[j] : (P.logscale ? exp10(x[nz + q]) : x[nz + q]);
    if (P.kscale) k *= P.kscale[(size_t)(i / P.Nch) * r + j];
    kr[j] = k;
  }
  __syncthreads();
  for (int idx = tid; idx < K * n; idx += DEF_BS) {
    const int m = idx / n, s = idx - m * n;
    double l[NPMAX], dl[NPMAX];
    lagrange(P, 0.5 * (P.tau[m] + P.tau[m + 1]), l, dl);
    double v = 0.0, d = 0.0;
    for (int j = 0; j < np; ++j) {
      v += l[j] * ze[j * n + s];
      d += dl[j] * ze[j * n + s];
    }
    zt[idx] = v;
    dz[idx] = d;
  }
  __syncthreads();
  for (int idx = tid; idx < K * r; idx += DEF_BS) {
    const int m = idx / r, j = idx - m * r;
    const int a = P.react[2 * j], b = P.react[2 * j + 1];
    double mo = kr[j] * zt[m * n + a];
    if (b >= 0) mo *= zt[m * n + b];
    mon[idx] = mo;
  }
  __syncthreads();
  double mx = 0.0;
  for (int idx = tid; idx < K * n; idx += DEF_BS) {
    const int m = idx / n, s = idx - m * n;
    double f = 0.0;
    for (int e = P.nu_ptr[s]; e < P.nu_ptr[s + 1]; ++e) f += P.nu_v[e] * mon[m * r + P.nu_r[e]];
    mx = fmax(mx, fabs(dz[idx] - P.h * f));
  }
  red[tid] = mx;
  __syncthreads();
  for (int w = DEF_BS / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] = fmax(red[tid], red[tid + w]);
    __syncthreads();
  }
  if (tid == 0) def[i] = red[0];
}

// Fine-mesh states from the coarse solution: one thread per (fine element,
// point, species).  In each experimental condition, time t = (i + tau_j) h_f
// (i the element within the condition) lies in the condition's coarse element
// ceil(t / h_c) - 1 (clamped; a time on a coarse boundary belongs to the left
// element, t = 0 to the first), at tau_c = t / h_c - i_c.
__global__ void k_interp(DevProb C, const double* __restrict__ xc, DevProb F,
                         double* __restrict__ xf) {
  const size_t nzf = (size_t)F.N * F.np * F.n;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nzf + F.p) return;
  if (idx >= nzf) {   // theta
    xf[idx] = xc[(size_t)C.N * C.np * C.n + (idx - nzf)];
    return;
  }
  const int n = F.n, s = (int)(idx % n);
  const size_t ij = idx / n;
  const int j = (int)(ij % F.np), ie = (int)(ij / F.np);
  const int cond = ie / F.Nch, i = ie - cond * F.Nch;
  const double t = ((double)i + F.tau[j]) * F.h;
  const double u = t / C.h;
  int ic = (int)ceil(u) - 1;
  ic = ic < 0 ? 0 : (ic > C.Nch - 1 ? C.Nch - 1 : ic);
  const double tc = u - ic;
  double l[NPMAX];
  lagrange(C, tc, l, nullptr);
  const size_t ec = (size_t)cond * C.Nch + ic;
  double v = 0.0;
  for (int a = 0; a < C.np; ++a) v += l[a] * xc[(ec * C.np + a) * n + s];
  xf[idx] = v;
}

__global__ void __launch_bounds__(DEF_BS) k_max(const double* __restrict__ v, int n,
                                                double* __restrict__ out) {
  __shared__ double red[DEF_BS];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += DEF_BS) m = fmax(m, v[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = DEF_BS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

static size_t defect_smem(const DevProb& P) {
  return sizeof(double) * ((size_t)P.np * P.n + 2 * (size_t)P.K * P.n + P.r + (size_t)P.K * P.r);
}

// Defect of x (device, n_x) into def (device, N) and its maximum into *mx
// (device); on the problem's stream.
static cudaError_t launch_defect(collo_problem* pr, const double* x, double* def, double* mx) {
  const size_t sm = defect_smem(pr->P);
  if (sm > SMEM_OPTIN_ABOVE)
    cudaFuncSetAttribute(k_defect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  count_launch(2);
  k_defect<<<pr->P.N, DEF_BS, sm, pr->stream>>>(pr->P, x, def);
  k_max<<<1, DEF_BS, 0, pr->stream>>>(def, pr->P.N, mx);
  return cudaGetLastError();
}

// Device scratch of a problem for the refinement calls: [N] defects + [1] max.
static double* refine_scratch(collo_problem* pr) {
  if (!pr->refine_buf) pr->refine_buf = pr->arena.alloc<double>((size_t)pr->P.N + 8);
  return pr->refine_buf;
}

}  // namespace collo

using namespace collo;

extern "C" {

collo_status collo_problem_create_refined(const collo_problem* coarse, int N,
                                          collo_problem** out) {
  if (!coarse || !out || N < 1) { set_error("bad argument"); return COLLO_ERR_INVALID_ARG; }
  const HostInputs& h = coarse->host;
  collo_network net{};
  net.n_species = coarse->P.n;
  net.n_reactions = coarse->P.r;
  net.reactants = h.react.data();
  net.products = h.prod.data();
  net.param_index = h.pidx.data();
  net.k_fixed = h.kfix.data();
  net.log10_params = coarse->P.logscale;
  net.x0 = h.x0.data();
  net.n_params = coarse->P.p;
  net.theta_lo = h.lo.data();
  net.theta_hi = h.hi.data();
  collo_observables obs{(int)h.species.size(), h.species.data()};
  collo_data data{(int)h.t.size(), h.t.data(), h.observable.data(), h.y.data(), h.sigma.data()};
  collo_mesh mesh{coarse->P.T, N, coarse->P.K,
                  coarse->P.gauss ? COLLO_SCHEME_GAUSS : COLLO_SCHEME_RADAU};
  collo_problem_options o{};
  o.precision = coarse->precision;
  o.device = coarse->device;
  o.launch_mode = coarse->launch_mode;
  collo_conditions cond{h.n_conditions, h.cond_x0.data(),
                        h.cond_scale.empty() ? nullptr : h.cond_scale.data(),
                        h.obs_cond.empty() ? nullptr : h.obs_cond.data()};
  return collo_problem_create_conditions(&net, &obs, &data, &mesh, &cond, &o, out);
}

collo_status collo_defect(collo_problem* prob, const double* x, double* per_element,
                          double* max_defect) {
  if (!prob || !x) { set_error("NULL argument"); return COLLO_ERR_INVALID_ARG; }
  COLLO_CUDA(cudaSetDevice(prob->device));
  double* buf = refine_scratch(prob);
  if (!buf) { set_error("device allocation failed"); return COLLO_ERR_OOM; }
  cudaStream_t st = prob->stream;
  double* xd = prob->kvec_c;   // staging
  COLLO_CUDA(cudaMemcpyAsync(xd, x, prob->n_x * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(launch_defect(prob, xd, buf, buf + prob->P.N));
  if (per_element)
    COLLO_CUDA(cudaMemcpyAsync(per_element, buf, prob->P.N * sizeof(double), cudaMemcpyDefault,
                               st));
  double mx = 0.0;
  COLLO_CUDA(cudaMemcpyAsync(&mx, buf + prob->P.N, sizeof(double), cudaMemcpyDeviceToHost, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  if (max_defect) *max_defect = mx;
  return COLLO_OK;
}

collo_status collo_interpolate(collo_problem* coarse, const double* x_coarse, collo_problem* fine,
                               double* x_fine) {
  if (!coarse || !x_coarse || !fine || !x_fine) {
    set_error("NULL argument");
    return COLLO_ERR_INVALID_ARG;
  }
  if (coarse->device != fine->device || coarse->P.n != fine->P.n || coarse->P.p != fine->P.p ||
      coarse->P.T != fine->P.T || coarse->P.Nc != fine->P.Nc) {
    set_error("coarse and fine problems differ in more than their meshes");
    return COLLO_ERR_INVALID_ARG;
  }
  COLLO_CUDA(cudaSetDevice(fine->device));
  cudaStream_t st = fine->stream;
  if ((size_t)coarse->n_x > (size_t)(fine->n_x + fine->n_c)) {
    set_error("the fine mesh has fewer than half the coarse mesh's elements");
    return COLLO_ERR_INVALID_ARG;
  }
  double* xc = fine->kvec_r;   // staging of the coarse solution
  double* xf = fine->kvec_c;
  COLLO_CUDA(cudaMemcpyAsync(xc, x_coarse, coarse->n_x * sizeof(double), cudaMemcpyDefault, st));
  const size_t tot = (size_t)fine->n_x;
  count_launch();
  k_interp<<<ceil_div((long long)tot, 256), 256, 0, st>>>(coarse->P, xc, fine->P, xf);
  COLLO_CUDA(cudaGetLastError());
  COLLO_CUDA(cudaMemcpyAsync(x_fine, xf, fine->n_x * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  return COLLO_OK;
}

collo_status collo_problem_set_start(collo_problem* prob, const double* x, const double* lambda) {
  if (!prob) { set_error("NULL problem"); return COLLO_ERR_INVALID_ARG; }
  COLLO_CUDA(cudaSetDevice(prob->device));
  if (!x) { prob->has_start = false; return COLLO_OK; }
  if (!prob->start_x) {
    prob->start_x = prob->arena.alloc<double>(prob->n_x);
    prob->start_lam = prob->arena.alloc<double>(prob->n_c);
    if (!prob->start_x || !prob->start_lam) {
      set_error("device allocation failed");
      return COLLO_ERR_OOM;
    }
  }
  COLLO_CUDA(cudaMemcpyAsync(prob->start_x, x, prob->n_x * sizeof(double), cudaMemcpyDefault,
                             prob->stream));
  if (lambda)
    COLLO_CUDA(cudaMemcpyAsync(prob->start_lam, lambda, prob->n_c * sizeof(double),
                               cudaMemcpyDefault, prob->stream));
  else
    COLLO_CUDA(cudaMemsetAsync(prob->start_lam, 0, prob->n_c * sizeof(double), prob->stream));
  COLLO_CUDA(cudaStreamSynchronize(prob->stream));
  prob->has_start = true;
  return COLLO_OK;
}

collo_status collo_refine_solve(collo_problem* const* probs, int count, const double* const* theta0,
                                const collo_ipm_options* opts, double defect_tol, int max_levels,
                                int max_elements, collo_problem** finals, collo_result* results,
                                int* levels) {
  if (!probs || count < 1 || !theta0 || !finals || !results || !levels || max_levels < 0 ||
      !(defect_tol > 0)) {
    set_error("bad argument");
    return COLLO_ERR_INVALID_ARG;
  }
  std::vector<collo_problem*> cur(probs, probs + count);
  for (int i = 0; i < count; ++i) { finals[i] = probs[i]; levels[i] = 0; }
  collo_status s = collo_batch_solve(cur.data(), count, theta0, opts, results);
  if (s != COLLO_OK) return s;
  auto cleanup = [&]() {
    for (int i = 0; i < count; ++i)
      if (cur[i] != probs[i]) { collo_problem_destroy(cur[i]); cur[i] = probs[i]; }
  };
  for (int lev = 1; lev <= max_levels; ++lev) {
    std::vector<int> idx;
    std::vector<collo_problem*> fine;
    std::vector<const double*> th;
    for (int i = 0; i < count; ++i) {
      const int st = results[i].status;
      if (st != COLLO_OK && st != COLLO_ACCEPTABLE) continue;
      collo_problem* c = cur[i];
      const int Nf = 2 * c->P.Nch;   // elements per condition
      if (max_elements > 0 && Nf > max_elements) continue;
      double mx = 0.0;
      if ((s = collo_defect(c, c->x, nullptr, &mx)) != COLLO_OK) { cleanup(); return s; }
      if (!(mx > defect_tol)) continue;
      collo_problem* f = nullptr;
      if ((s = collo_problem_create_refined(c, Nf, &f)) != COLLO_OK) { cleanup(); return s; }
      // the interpolated solution is the fine problem's start (lambda = 0)
      double* xs = f->kvec_a;   // device scratch of n_x + n_c doubles
      if ((s = collo_interpolate(c, c->x, f, xs)) != COLLO_OK ||
          (s = collo_problem_set_start(f, xs, nullptr)) != COLLO_OK) {
        collo_problem_destroy(f);
        cleanup();
        return s;
      }
      idx.push_back(i);
      fine.push_back(f);
      th.push_back(f->start_x + (f->n_x - f->P.p));
    }
    if (idx.empty()) break;
    std::vector<collo_result> res(idx.size());
    for (size_t k = 0; k < idx.size(); ++k) {
      res[k] = collo_result{};
      res[k].theta = results[idx[k]].theta;   // theta keeps its size across meshes
    }
    s = collo_batch_solve(fine.data(), (int)fine.size(), th.data(), opts, res.data());
    if (s != COLLO_OK) {
      for (auto* f : fine) collo_problem_destroy(f);
      cleanup();
      return s;
    }
    for (size_t k = 0; k < idx.size(); ++k) {
      const int i = idx[k];
      if (cur[i] != probs[i]) collo_problem_destroy(cur[i]);
      cur[i] = fine[k];
      finals[i] = fine[k];
      results[i] = res[k];
      levels[i] = lev;
    }
  }
  return COLLO_OK;
}

}  // extern "C"
