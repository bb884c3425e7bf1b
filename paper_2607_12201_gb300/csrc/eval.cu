// Evaluation kernels: residuals, constraint Jacobian, Lagrangian Hessian and
// objective of the Radau-collocation NLP (paper Eq. 2 and Eq. 3), evaluated in
// parallel over every (element, node) pair -- the "single instruction,
// multiple data" evaluation the paper builds with ExaModels (Section
// "Constructing GPU kernels with ExaModels.jl"), written here as one CUDA
// block per element.  Also the structured FP64 KKT matrix-vector product used
// by iterative refinement and by the optimality test.
#include <mutex>

#include "collo_internal.cuh"
#include "resid.cuh"
#include "problem.cuh"

namespace collo {

cudaError_t launch_chunk_sums(const double* X, int C, int L, double* part, cudaStream_t st);


__device__ inline double sum_chunks(const double* __restrict__ part, int G, int L, int l) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int g = 0;
  for (; g + 3 < G; g += 4) {
    a0 += part[(size_t)g * L + l];
    a1 += part[(size_t)(g + 1) * L + l];
    a2 += part[(size_t)(g + 2) * L + l];
    a3 += part[(size_t)(g + 3) * L + l];
  }
  for (; g < G; ++g) a0 += part[(size_t)g * L + l];
  return (a0 + a1) + (a2 + a3);
}

// Observation weights l_j(tau_m) (Lagrange basis on the element's
// interpolation points) and the observation's element; one thread per
// observation.
__global__ void k_obs_weights(DevProb P, int M, int N, double T, const double* __restrict__ t,
                              int* __restrict__ elem, double* __restrict__ w) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double u = t[m] * N / T;
  int i = (int)ceil(u) - 1;
  i = i < 0 ? 0 : (i > N - 1 ? N - 1 : i);
  double tau = u - i;
  elem[m] = i;
  const int np = P.np;
  for (int j = 0; j < np; ++j) {
    double v = 1.0;
    for (int l = 0; l < np; ++l)
      if (l != j) v *= (tau - P.tau[l]) / (P.tau[j] - P.tau[l]);
    w[m * np + j] = v;
  }
}

// Rate constant of reaction j and its first and second theta derivatives.
__device__ inline void rate_const(const DevProb& P, int j, const double* x, const double* dx,
                                  double alpha, double& k, double& dk, double& d2k) {
  int q = P.pidx[j];
  if (q < 0) {
    k = P.kfix[j]; dk = 0.0; d2k = 0.0;
    return;
  }
  size_t o = (size_t)P.N * P.np * P.n + q;
  double th = x[o];
  if (dx) th += alpha * dx[o];
  if (P.logscale) {
    const double ln10 = 2.302585092994045684;
    k = exp10(th);
    dk = ln10 * k;
    d2k = ln10 * ln10 * k;
  } else {
    k = th; dk = 1.0; d2k = 0.0;
  }
}

// One block per element i.  Evaluates at x + alpha dx (dx may be null).
// DERIV = false: residuals, objective and norms only (line-search trials).
template <bool DERIV>
__device__ void eval_elem(const DevProb& P, const double* __restrict__ x,
                          const double* __restrict__ dx, double alpha,
                          const double* __restrict__ lam, double obj_factor, const DevEval& E,
                          int i, double* sm, double* red) {
  const int n = P.n, r = P.r, p = P.p, K = P.K, np = P.np;
  const int tid = threadIdx.x;
  double* ze = sm;              // [K+1][n]
  double* le = ze + np * n;     // [K+1][n]
  double* kr = le + np * n;     // [r]
  double* dkr = kr + r;         // [r]
  double* d2kr = dkr + r;       // [r]
  double* mon = d2kr + r;       // [K][r]
  double* da = mon + K * r;     // [K][r] d mon / d z(slot 0)
  double* db = da + K * r;      // [K][r] d mon / d z(slot 1)
  double* om = db + K * r;      // [K][r] sum_s lambda_s nu_s,r
  const size_t zoff = (size_t)i * np * n;

  for (int t = tid; t < np * n; t += EVAL_BS) {
    double v = x[zoff + t];
    if (dx) v += alpha * dx[zoff + t];
    ze[t] = v;
    le[t] = (DERIV && lam) ? lam[zoff + t] : 0.0;
  }
  for (int j = tid; j < r; j += EVAL_BS) {
    rate_const(P, j, x, dx, alpha, kr[j], dkr[j], d2kr[j]);
    if (P.kscale) {   // the element's condition input (lifted p^c, Eq. 3)
      const double u = P.kscale[(size_t)(i / P.Nch) * r + j];
      kr[j] *= u; dkr[j] *= u; d2kr[j] *= u;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < K * r; idx += EVAL_BS) {
    const int k = idx / r + 1, j = idx - (idx / r) * r;
    const int a = P.react[2 * j], b = P.react[2 * j + 1];
    const double za = ze[k * n + a];
    double mo, dA, dB;
    if (b < 0) { mo = za; dA = 1.0; dB = 0.0; }
    else { const double zb = ze[k * n + b]; mo = za * zb; dA = zb; dB = za; }
    mon[idx] = mo; da[idx] = dA; db[idx] = dB;
    if (DERIV) {
      double o = -le[k * n + a];
      if (b >= 0) o -= le[k * n + b];
      const int p0 = P.prod[2 * j], p1 = P.prod[2 * j + 1];
      if (p0 >= 0) o += le[k * n + p0];
      if (p1 >= 0) o += le[k * n + p1];
      om[idx] = o;
    }
  }
  __syncthreads();

  // constraints: continuity / initial (point 0) and collocation (points 1..K)
  double csum = 0.0, cmax = 0.0;
  for (int idx = tid; idx < np * n; idx += EVAL_BS) {
    const int j = idx / n, s = idx - j * n;
    double c;
    if (j == 0) {
      double prev;
      if (!chain_start(P, i) && !P.gauss) {   // Radau: b_j = delta_jK
        prev = x[zoff - n + s];
        if (dx) prev += alpha * dx[zoff - n + s];
      } else if (!chain_start(P, i)) {        // Gauss: sum_j b_j z[i-1][j]
        const size_t po = zoff - (size_t)np * n + s;
        prev = 0.0;
        for (int jj = 0; jj < np; ++jj) {
          double v = x[po + (size_t)jj * n];
          if (dx) v += alpha * dx[po + (size_t)jj * n];
          prev += P.bw[jj] * v;
        }
      } else {   // initial condition of the element's experimental condition
        prev = P.x0[(size_t)(i / P.Nch) * n + s];
      }
      c = ze[s] - prev;
    } else {
      double acc = 0.0;
      for (int jj = 0; jj < np; ++jj) acc += P.D[j][jj] * ze[jj * n + s];
      double f = 0.0;
      for (int e = P.nu_ptr[s]; e < P.nu_ptr[s + 1]; ++e) {
        const int rr = P.nu_r[e];
        f += P.nu_v[e] * kr[rr] * mon[(j - 1) * r + rr];
      }
      c = acc - P.h * f;
    }
    E.c[zoff + idx] = c;
    csum += fabs(c);
    cmax = fmax(cmax, fabs(c));
  }

  // objective terms of this element's observations
  const int o0 = P.obs_ptr[i], o1 = P.obs_ptr[i + 1];
  double phi = 0.0;
  for (int o = o0 + tid; o < o1; o += EVAL_BS) {
    const int s = P.obs_s[o];
    double yh = 0.0;
    for (int j = 0; j < np; ++j) yh += P.obs_w[o * np + j] * ze[j * n + s];
    const double res = (yh - P.obs_y[o]) / P.obs_sig[o];
    phi += 0.5 * res * res;
  }
  phi = block_sum<EVAL_BS>(phi, red);
  csum = block_sum<EVAL_BS>(csum, red);
  cmax = block_max<EVAL_BS>(cmax, red);
  if (tid == 0) {
    E.part[i * 4 + 0] = phi;
    E.part[i * 4 + 1] = csum;
    E.part[i * 4 + 2] = cmax;
    E.part[i * 4 + 3] = 0.0;
  }
  if (!DERIV) return;

  // gradient of obj_factor * Phi with respect to z[i][j][s]
  for (int idx = tid; idx < np * n; idx += EVAL_BS) {
    const int j = idx / n, s = idx - j * n;
    double g = 0.0;
    for (int o = o0; o < o1; ++o) {
      if (P.obs_s[o] != s) continue;
      double yh = 0.0;
      for (int jj = 0; jj < np; ++jj) yh += P.obs_w[o * np + jj] * ze[jj * n + s];
      const double sg = P.obs_sig[o];
      g += P.obs_w[o * np + j] * (yh - P.obs_y[o]) / (sg * sg);
    }
    E.grad[zoff + idx] = obj_factor * g;
  }
  if (i == 0)
    for (int q = tid; q < p; q += EVAL_BS) E.grad[(size_t)P.N * np * n + q] = 0.0;
  // objective Hessian blocks Wobj[i][s][j][l]
  const int np2 = np * np;
  for (int idx = tid; idx < n * np2; idx += EVAL_BS) {
    const int s = idx / np2, j = (idx / np) % np, l = idx % np;
    double w = 0.0;
    for (int o = o0; o < o1; ++o) {
      if (P.obs_s[o] != s) continue;
      const double sg = P.obs_sig[o];
      w += P.obs_w[o * np + j] * P.obs_w[o * np + l] / (sg * sg);
    }
    E.Wobj[(size_t)i * n * np2 + idx] = obj_factor * w;
  }
  const double mh = -P.h;
  // Derivative blocks, one thread per row.  Row s of JZ / JT at node k
  // accumulates, over the reactions r changing species s (nu[s][r] != 0),
  // -h nu k_r dmon_r/dz (into the reactant columns) and -h nu dk_r mon_r
  // (into column pidx[r]).  Row t of Wzz / Wzt at node k accumulates, over the
  // reactions consuming t, -h om_r k_r d2mon_r/dz_t dz_u and
  // -h om_r dk_r dmon_r/dz_t.  Each row is owned by one thread (fixed order).
  for (int idx = tid; idx < K * n; idx += EVAL_BS) {
    const int k = idx / n + 1, s = idx - (k - 1) * n;
    double* jz = E.JZ + (((size_t)i * K + (k - 1)) * n + s) * n;
    double* jt = E.JT + (((size_t)i * K + (k - 1)) * n + s) * p;
    for (int t = 0; t < n; ++t) jz[t] = 0.0;
    for (int q = 0; q < p; ++q) jt[q] = 0.0;
    for (int e = P.nu_ptr[s]; e < P.nu_ptr[s + 1]; ++e) {
      const int rr = P.nu_r[e];
      const int a = P.react[2 * rr], b = P.react[2 * rr + 1];
      const int mi = (k - 1) * r + rr;
      const double c = mh * P.nu_v[e];
      jz[a] += c * kr[rr] * da[mi];
      if (b >= 0) jz[b] += c * kr[rr] * db[mi];
      const int q = P.pidx[rr];
      if (q >= 0) jt[q] += c * dkr[rr] * mon[mi];
    }
  }
  for (int idx = tid; idx < K * n; idx += EVAL_BS) {
    const int k = idx / n + 1, t = idx - (k - 1) * n;
    double* wz = E.Wzz + (((size_t)i * K + (k - 1)) * n + t) * n;
    double* wt = E.Wzt + (((size_t)i * K + (k - 1)) * n + t) * p;
    for (int u = 0; u < n; ++u) wz[u] = 0.0;
    for (int q = 0; q < p; ++q) wt[q] = 0.0;
    for (int e = P.rs_ptr[t]; e < P.rs_ptr[t + 1]; ++e) {
      const int rr = P.rs_r[e];
      const int a = P.react[2 * rr], b = P.react[2 * rr + 1];
      const int mi = (k - 1) * r + rr;
      const double c = mh * om[mi];
      if (b >= 0) {
        if (a == b) wz[t] += c * kr[rr] * 2.0;
        else wz[a == t ? b : a] += c * kr[rr];
      }
      const int q = P.pidx[rr];
      if (q >= 0) {
        double dm = 0.0;
        if (a == t) dm += da[mi];
        if (b == t) dm += db[mi];
        wt[q] += c * dkr[rr] * dm;
      }
    }
  }
  // theta-theta diagonal partial sums of this element
  for (int q = tid; q < p; q += EVAL_BS) {
    double v = 0.0;
    for (int k = 1; k <= K; ++k)
      for (int e = P.pr_ptr[q]; e < P.pr_ptr[q + 1]; ++e) {
        const int rr = P.pr_r[e];
        const int mi = (k - 1) * r + rr;
        v += om[mi] * d2kr[rr] * mon[mi];
      }
    E.wtt_part[(size_t)i * p + q] = mh * v;
  }
}

template <bool DERIV>
__global__ void __launch_bounds__(EVAL_BS)
k_eval(DevProb P, const double* __restrict__ x, const double* __restrict__ dx, double alpha,
       const double* __restrict__ lam, double obj_factor, DevEval E) {
  extern __shared__ double sm[];
  __shared__ double red[EVAL_BS];
  eval_elem<DERIV>(P, x, dx, alpha, lam, obj_factor, E, blockIdx.x, sm, red);
}

// Vector selectors of the batched kernels (which per-instance array to use).
enum VecSel { V_NONE = 0, V_X = 1, V_LAM = 2, V_STAGE_X = 3, V_STAGE_L = 4, V_KB = 5 };

__device__ inline const double* pick_vec(const DevInst& I, int sel) {
  switch (sel) {
    case V_X: return I.x;
    case V_LAM: return I.lam;
    case V_STAGE_X: return I.kc;
    case V_STAGE_L: return I.kc + I.n_x;
    case V_KB: return I.kb;
    default: return nullptr;
  }
}

// Batched evaluation: block t evaluates element t - pre[k] of instance act[k]
// at x + alpha_k dx.
template <bool DERIV>
__global__ void __launch_bounds__(EVAL_BS)
k_eval_b(const DevInst* __restrict__ insts, const int* __restrict__ act, int A,
         const int* __restrict__ pre, const InstParams* __restrict__ prm, int xsel, int dxsel,
         int lsel) {
  extern __shared__ double sm[];
  __shared__ double red[EVAL_BS];
  const int t = blockIdx.x;
  const int k = find_item(pre, A, t);
  const DevInst& I = insts[act[k]];
  eval_elem<DERIV>(I.P, pick_vec(I, xsel), pick_vec(I, dxsel), prm[k].alpha, pick_vec(I, lsel),
                   prm[k].obj_factor, I.E, t - pre[k], sm, red);
}

// Sum the per-element partials in a fixed order: phi, |c|_1, |c|_inf, W_thth.
__device__ void eval_reduce_one(const DevProb& P, const DevEval& E, int deriv, double* out,
                                double* sh) {
  const int tid = threadIdx.x;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = tid; i < P.N; i += RED_BS) {
    a += E.part[i * 4 + 0];
    b += E.part[i * 4 + 1];
    c = fmax(c, E.part[i * 4 + 2]);
  }
  a = block_sum<RED_BS>(a, sh);
  b = block_sum<RED_BS>(b, sh);
  c = block_max<RED_BS>(c, sh);
  if (tid == 0) {
    E.red[0] = a; E.red[1] = b; E.red[2] = c;
    if (out) { out[O_PHI] = a; out[O_C1] = b; out[O_CINF] = c; }
  }
  if (!deriv) return;
  // W_thth: warp w sums column q over elements lane, lane + 32, ... then a
  // fixed shuffle tree
  const int lane = tid & 31, warp = tid >> 5;
  for (int q = warp; q < P.p; q += RED_BS / 32) {
    double v = 0.0;
    for (int i = lane; i < P.N; i += 32) v += E.wtt_part[(size_t)i * P.p + q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) E.wtt[q] = v;
  }
}

__global__ void __launch_bounds__(RED_BS) k_eval_reduce(DevProb P, DevEval E, int deriv) {
  __shared__ double sh[RED_BS];
  eval_reduce_one(P, E, deriv, nullptr, sh);
}

// Reduction of collo_eval_noalloc: the partials in the fixed scratch, Phi
// into the caller's output (out[0] = Phi).
__global__ void __launch_bounds__(RED_BS) k_eval_reduce_noalloc(DevProb P, DevEval E, double* phi) {
  __shared__ double sh[RED_BS];
  eval_reduce_one(P, E, 1, nullptr, sh);
  if (threadIdx.x == 0) *phi = E.red[0];
}

__global__ void __launch_bounds__(RED_BS)
k_eval_reduce_b(const DevInst* __restrict__ insts, const int* __restrict__ act, int deriv) {
  __shared__ double sh[RED_BS];
  const DevInst& I = insts[act[blockIdx.x]];
  eval_reduce_one(I.P, I.E, deriv, I.out, sh);
}

__global__ void __launch_bounds__(EVAL_BS)
k_kkt_resid(DevProb P, DevEval E, const double* __restrict__ sigma, double dw, double dc,
            const double* __restrict__ vx, const double* __restrict__ vl,
            const double* __restrict__ bx, double bxs, const double* __restrict__ bc, double bcs,
            double* __restrict__ rout, double* __restrict__ thpart, double* __restrict__ npart) {
  __shared__ double red[EVAL_BS];
  resid_elem(P, E, sigma, dw, dc, vx, vl, bx, bxs, bc, bcs, rout, thpart, npart, blockIdx.x, red);
}

// BS: 64 when every instance of the batch has at most 64 state rows per
// element ((K + 1) n), else EVAL_BS; the results do not depend on it.
template <int BS>
__global__ void __launch_bounds__(BS)
k_kkt_resid_b(const DevInst* __restrict__ insts, const int* __restrict__ act, int A,
              const int* __restrict__ pre, const InstParams* __restrict__ prm, int mode) {
  __shared__ double red[BS];
  const int t = blockIdx.x;
  const int k = find_item(pre, A, t);
  const DevInst& I = insts[act[k]];
  const ResidArgs a = resid_args(I, prm[k], mode);
  resid_elem<BS>(I.P, I.E, a.sigma, a.dw, a.dc, a.vx, a.vl, a.bx, a.bxs, a.bc, a.bcs, a.rout,
                 I.thpart, I.npart, t - pre[k], red);
}

__global__ void __launch_bounds__(RED_BS)
k_kkt_resid_theta(DevProb P, DevEval E, const double* __restrict__ sigma, double dw,
                  const double* __restrict__ vx, const double* __restrict__ bx, double bxs,
                  const double* __restrict__ bc, double* __restrict__ rout,
                  const double* __restrict__ thpart, const double* __restrict__ npart,
                  const double* __restrict__ th_extra, double* __restrict__ out) {
  __shared__ double sh[RED_BS];
  resid_theta_one(P, E, sigma, dw, vx, bx, bxs, bc, rout, thpart, npart, th_extra, out, sh);
}

__global__ void __launch_bounds__(RED_BS)
k_kkt_resid_theta_b(const DevInst* __restrict__ insts, const int* __restrict__ act,
                    const InstParams* __restrict__ prm, int mode) {
  __shared__ double sh[RED_BS];
  const int k = blockIdx.x;
  const DevInst& I = insts[act[k]];
  const ResidArgs a = resid_args(I, prm[k], mode);
  resid_theta_one(I.P, I.E, a.sigma, a.dw, a.vx, a.bx, a.bxs, a.bc, a.rout, I.thpart, I.npart,
                  a.th_extra, I.out + O_RX, sh);
}

// ---- host launchers -------------------------------------------------------------
size_t eval_smem_bytes(const DevProb& P) {
  return sizeof(double) * (size_t)(2 * P.np * P.n + 3 * P.r + 4 * P.K * P.r);
}

cudaError_t launch_obs_weights(const DevProb& P, int M, int N, double T, const double* t,
                               int* elem, double* w, cudaStream_t st) {
  if (M == 0) return cudaSuccess;
  count_launch();
  k_obs_weights<<<ceil_div(M, 128), 128, 0, st>>>(P, M, N, T, t, elem, w);
  return cudaGetLastError();
}

cudaError_t launch_eval(const DevProb& P, const DevEval& E, const double* x, const double* dx,
                        double alpha, const double* lam, double obj_factor, bool deriv,
                        cudaStream_t st) {
  size_t sm = eval_smem_bytes(P);
  if (deriv) {
    if (sm > SMEM_OPTIN_ABOVE)
      cudaFuncSetAttribute(k_eval<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    count_launch();
    k_eval<true><<<P.N, EVAL_BS, sm, st>>>(P, x, dx, alpha, lam, obj_factor, E);
  } else {
    if (sm > SMEM_OPTIN_ABOVE)
      cudaFuncSetAttribute(k_eval<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    count_launch();
    k_eval<false><<<P.N, EVAL_BS, sm, st>>>(P, x, dx, alpha, lam, obj_factor, E);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  k_eval_reduce<<<1, RED_BS, 0, st>>>(P, E, deriv ? 1 : 0);
  return cudaGetLastError();
}

// r = [bxs bx; bcs bc] - K [vx; vl] (null vectors are zero; th_extra, if given,
// is subtracted from the parameter rows of K v).  out[0..2] = max|r_x|,
// max|r_c|, max|b|.  rout may be null (norms only).
cudaError_t launch_kkt_resid(const DevProb& P, const DevEval& E, const double* sigma, double dw,
                             double dc, const double* vx, const double* vl, const double* bx,
                             double bxs, const double* bc, double bcs, double* rout,
                             double* thpart, double* npart, const double* th_extra, double* out,
                             cudaStream_t st) {
  count_launch();
  k_kkt_resid<<<P.N, EVAL_BS, 0, st>>>(P, E, sigma, dw, dc, vx, vl, bx, bxs, bc, bcs, rout,
                                       thpart, npart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  k_kkt_resid_theta<<<1, RED_BS, 0, st>>>(P, E, sigma, dw, vx, bx, bxs, bc, rout, thpart, npart,
                                          th_extra, out);
  return cudaGetLastError();
}

// ---- evaluation without allocation ------------------------------------------------
// Callers that cannot allocate device memory while running (real-time control
// loops that allocate everything up front so that no call can fail or stall on
// an allocation, hosts whose device allocator is owned by another runtime or
// memory pool) use collo_eval_noalloc.
// Its only scratch, the per-element partial sums of the objective, of the
// constraint norms and of the parameter-parameter Hessian, lives in this
// fixed device array instead of problem-owned buffers.  Every GPU that loads
// the library holds it until the process exits.
constexpr size_t NOALLOC_SCRATCH_DOUBLES = 1 << 19;   // 4 MiB
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];   // device address of the array, per device ordinal

// Device address of the scratch array on device `dev` (current device).
// cudaGetSymbolAddress runs once per device, at the first call there (which
// therefore belongs before any stream capture on that device); in host code
// the array's name is only a host-side stand-in and must never be passed to a
// kernel.
static cudaError_t noalloc_scratch(int dev, double** out) {
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = ptr;
  }
  *out = static_cast<double*>(g_noalloc_addr[dev]);
  return cudaSuccess;
}

// ---- batched launchers (plan arrays in device memory) --------------------------
cudaError_t launch_eval_b(const DevInst* insts, const int* act, int A, const int* pre_elem,
                          int total_elems, const InstParams* prm, int xsel, int dxsel, int lsel,
                          bool deriv, size_t smem, cudaStream_t st) {
  if (A == 0) return cudaSuccess;
  if (deriv) {
    if (smem > SMEM_OPTIN_ABOVE)
      cudaFuncSetAttribute(k_eval_b<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launch();
    k_eval_b<true><<<total_elems, EVAL_BS, smem, st>>>(insts, act, A, pre_elem, prm, xsel, dxsel, lsel);
  } else {
    if (smem > SMEM_OPTIN_ABOVE)
      cudaFuncSetAttribute(k_eval_b<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launch();
    k_eval_b<false><<<total_elems, EVAL_BS, smem, st>>>(insts, act, A, pre_elem, prm, xsel, dxsel, lsel);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  k_eval_reduce_b<<<A, RED_BS, 0, st>>>(insts, act, deriv ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_resid_b(const DevInst* insts, const int* act, int A, const int* pre_elem,
                           int total_elems, int max_n, const InstParams* prm, int mode,
                           cudaStream_t st) {
  if (A == 0) return cudaSuccess;
  count_launch();
  if (max_n <= 64)
    k_kkt_resid_b<64><<<total_elems, 64, 0, st>>>(insts, act, A, pre_elem, prm, mode);
  else
    k_kkt_resid_b<EVAL_BS><<<total_elems, EVAL_BS, 0, st>>>(insts, act, A, pre_elem, prm, mode);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  k_kkt_resid_theta_b<<<A, RED_BS, 0, st>>>(insts, act, prm, mode);
  return cudaGetLastError();
}

}  // namespace collo

// ---- C ABI: evaluation without allocation -------------------------------------------

namespace {
// Restores the caller's current device when the call returns.
struct DeviceRestore {
  int dev = -1;
  DeviceRestore() {
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = -1; }
  }
  ~DeviceRestore() {
    if (dev >= 0) cudaSetDevice(dev);
  }
};
// True when p is device (or managed) memory of device `dev`; a host pointer,
// pinned or pageable, or memory of another GPU is refused.  Allocates nothing.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}
}  // namespace

extern "C" collo_status collo_eval_noalloc(collo_problem* prob, const double* x,
                                           const double* lambda, double obj_factor,
                                           const collo_eval_out* out, void* stream) {
  using namespace collo;
  if (!prob || !x || !out || !out->phi || !out->c || !out->grad || !out->jac_z ||
      !out->jac_theta || !out->hess_zz || !out->hess_ztheta || !out->hess_obj ||
      (prob->P.p > 0 && !out->hess_thth)) {
    set_error("collo_eval_noalloc: x and every output must be device pointers (lambda may be NULL)");
    return COLLO_ERR_INVALID_ARG;
  }
  DeviceRestore restore;
  {
    const void* ptrs[] = {x, lambda, out->phi, out->c, out->grad, out->jac_z, out->jac_theta,
                          out->hess_zz, out->hess_ztheta, out->hess_obj, out->hess_thth};
    const char* names[] = {"x", "lambda", "phi", "c", "grad", "jac_z", "jac_theta", "hess_zz",
                           "hess_ztheta", "hess_obj", "hess_thth"};
    for (int k = 0; k < 11; ++k) {
      if (!ptrs[k]) continue;   // lambda, or hess_thth with p = 0
      if (!on_device(ptrs[k], prob->device)) {
        set_error(std::string("collo_eval_noalloc: ") + names[k] +
                  " is not device memory of the problem's GPU");
        return COLLO_ERR_INVALID_ARG;
      }
    }
  }
  const DevProb& P = prob->P;
  const size_t need = (size_t)P.N * (4 + (size_t)P.p) + 8;
  if (need > NOALLOC_SCRATCH_DOUBLES) {
    set_error("collo_eval_noalloc: N (4 + p) + 8 = " + std::to_string(need) +
              " doubles exceeds the fixed scratch of " +
              std::to_string(NOALLOC_SCRATCH_DOUBLES) + " doubles");
    return COLLO_ERR_INVALID_ARG;
  }
  COLLO_CUDA(cudaSetDevice(prob->device));
  double* scratch = nullptr;
  COLLO_CUDA(noalloc_scratch(prob->device, &scratch));
  DevEval E{};
  E.c = out->c;
  E.grad = out->grad;
  E.JZ = out->jac_z;
  E.JT = out->jac_theta;
  E.Wzz = out->hess_zz;
  E.Wzt = out->hess_ztheta;
  E.Wobj = out->hess_obj;
  E.wtt = out->hess_thth;
  E.part = scratch;                                   // [N][4]
  E.wtt_part = scratch + (size_t)P.N * 4;             // [N][p]
  E.red = scratch + (size_t)P.N * (4 + (size_t)P.p);  // [8]
  cudaStream_t st = stream ? (cudaStream_t)stream : prob->stream;
  const size_t sm = eval_smem_bytes(P);
  if (sm > SMEM_OPTIN_ABOVE)
    COLLO_CUDA(cudaFuncSetAttribute(k_eval<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  count_launch();
  k_eval<true><<<P.N, EVAL_BS, sm, st>>>(P, x, nullptr, 0.0, lambda, obj_factor, E);
  COLLO_CUDA(cudaGetLastError());
  count_launch();
  k_eval_reduce_noalloc<<<1, RED_BS, 0, st>>>(P, E, out->phi);
  COLLO_CUDA(cudaGetLastError());
  return COLLO_OK;
}
