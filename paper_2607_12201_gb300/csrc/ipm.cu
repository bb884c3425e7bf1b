// Filter line-search primal-dual interior-point driver (paper Introduction:
// the NLP is solved by "a filter line-search interior point solver"; the
// algorithm statement followed is Waechter & Biegler, 2006) with every
// iterate resident on the device, and the collocation forward sweep that
// gives its initial states (paper Section "Optimization framework
// configurations": initial guesses from a forward solve at theta0).
//
// The host runs only scalar control (filter, barrier and inertia-correction
// decisions); vectors never leave the GPU.  Per iteration the host reads one
// small block of scalars after each phase.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "problem.cuh"

namespace collo {

constexpr int IBS = 256;

template <int BS>
__device__ double bsum(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = BS / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}
template <int BS>
__device__ double bmax(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = BS / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] = fmax(sh[t], sh[t + s]);
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}
template <int BS>
__device__ double bmin(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = BS / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] = fmin(sh[t], sh[t + s]);
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, double a, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

cudaError_t launch_axpy(double* y, const double* x, double a, size_t n, cudaStream_t st) {
  int g = (int)std::min<size_t>((n + 255) / 256, 4096);
  count_launch();
  k_axpy<<<std::max(g, 1), 256, 0, st>>>(y, x, a, n);
  return cudaGetLastError();
}

// Two-stage deterministic reductions: partial[b] over a grid-stride slice.
constexpr int RGRID = 256;
__global__ void __launch_bounds__(IBS) k_dot_part(const double* __restrict__ a,
                                                  const double* __restrict__ b, size_t n,
                                                  int absmode, double* __restrict__ part) {
  __shared__ double sh[IBS];
  double v = 0.0;
  for (size_t i = blockIdx.x * (size_t)IBS + threadIdx.x; i < n; i += (size_t)RGRID * IBS)
    v += absmode ? fabs(a[i]) : a[i] * b[i];
  v = bsum<IBS>(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}
__global__ void __launch_bounds__(IBS) k_sum_parts(const double* __restrict__ part,
                                                   double* __restrict__ out) {
  __shared__ double sh[IBS];
  double v = 0.0;
  for (int i = threadIdx.x; i < RGRID; i += IBS) v += part[i];
  v = bsum<IBS>(v, sh);
  if (threadIdx.x == 0) *out = v;
}

// theta0 pushed into the bounds (Waechter & Biegler 2006, Sec. 3.6), bound
// duals 1.
__global__ void k_init_point(DevProb P, const double* __restrict__ theta0, double* __restrict__ x,
                             double* __restrict__ zl, double* __restrict__ zu, double kappa1,
                             double kappa2) {
  const size_t nz = (size_t)P.N * NP * P.n;
  for (int q = threadIdx.x; q < P.p; q += blockDim.x) {
    const double lo = P.theta_lo[q], hi = P.theta_hi[q];
    const double pl = fmin(kappa1 * fmax(1.0, fabs(lo)), kappa2 * (hi - lo));
    const double pu = fmin(kappa1 * fmax(1.0, fabs(hi)), kappa2 * (hi - lo));
    x[nz + q] = fmin(fmax(theta0[q], lo + pl), hi - pu);
    zl[q] = 1.0;
    zu[q] = 1.0;
  }
}

// Collocation forward sweep at theta = x[nz..]: for each element in turn,
// Newton's method on the K collocation equations in the element's interior
// states, started at the element's initial state, stopped when
// max|dZ| <= 1e-12 max(1, max|Z|) (at most 30 iterations); an element whose
// iteration fails keeps the constant guess.  The residual, the update and
// the stopping test are FP64; the Newton correction solves the Jacobian
// system by FP32 LU with partial pivoting (an inexact Newton step whose
// error the FP64 residual of the next iteration corrects), so the sweep
// converges to the same FP64 collocation solution.  One block of SWEEP_BS
// threads; the FP32 augmented matrix [J | G] sits in shared memory, or in
// gwork when 3n is too large.
constexpr int SWEEP_MAXIT = 30;
constexpr int SWEEP_BS = 256;
__global__ void __launch_bounds__(SWEEP_BS) k_forward_sweep(DevProb P, double* __restrict__ x,
                                                            int* __restrict__ fails,
                                                            float* __restrict__ gwork) {
  extern __shared__ double sm[];
  __shared__ int s_piv;
  __shared__ float s_inv;
  __shared__ double s_red[SWEEP_BS];
  __shared__ int s_flag;
  const int n = P.n, r = P.r, dim = KC * n, ldj = dim + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* kr = sm;                 // [r]
  double* mon = kr + r;            // [3][r]
  double* da = mon + KC * r;       // [3][r]
  double* db = da + KC * r;        // [3][r]
  double* z0 = db + KC * r;        // [n]
  double* Z = z0 + n;              // [3n]
  double* dZ = Z + dim;            // [3n]
  float* Jm = gwork ? gwork : reinterpret_cast<float*>(dZ + dim);  // [dim][dim+1]
  const size_t nz = (size_t)P.N * NP * n;
  for (int j = tid; j < r; j += SWEEP_BS) {
    const int q = P.pidx[j];
    if (q < 0) kr[j] = P.kfix[j];
    else kr[j] = P.logscale ? exp10(x[nz + q]) : x[nz + q];
  }
  for (int s = tid; s < n; s += SWEEP_BS) z0[s] = P.x0[s];
  __syncthreads();
  int nfail = 0;
  for (int i = 0; i < P.N; ++i) {
    for (int t = tid; t < dim; t += SWEEP_BS) Z[t] = z0[t % n];
    __syncthreads();
    bool ok = false;
    for (int it = 0; it < SWEEP_MAXIT; ++it) {
      for (int idx = tid; idx < KC * r; idx += SWEEP_BS) {
        const int k = idx / r, j = idx - k * r;
        const int a = P.react[2 * j], b = P.react[2 * j + 1];
        const double za = Z[k * n + a];
        if (b < 0) { mon[idx] = za; da[idx] = 1.0; db[idx] = 0.0; }
        else { const double zb = Z[k * n + b]; mon[idx] = za * zb; da[idx] = zb; db[idx] = za; }
      }
      __syncthreads();
      // Jacobian entries D[k][j] delta_st - delta_kj h df_s/dz_t, and G (FP64)
      for (int idx = tid; idx < dim * dim; idx += SWEEP_BS) {
        const int row = idx / dim, col = idx - row * dim;
        const int k = row / n + 1, s = row - (k - 1) * n;
        const int j = col / n + 1, t = col - (j - 1) * n;
        double v = (s == t) ? P.D[k][j] : 0.0;
        if (j == k) {
          double fz = 0.0;
          for (int e = P.nu_ptr[s]; e < P.nu_ptr[s + 1]; ++e) {
            const int rr = P.nu_r[e];
            const int a = P.react[2 * rr], b = P.react[2 * rr + 1];
            const int mi = (k - 1) * r + rr;
            double dm = 0.0;
            if (a == t) dm += da[mi];
            if (b == t) dm += db[mi];
            fz += P.nu_v[e] * kr[rr] * dm;
          }
          v -= P.h * fz;
        }
        Jm[(size_t)row * ldj + col] = (float)v;
      }
      for (int row = tid; row < dim; row += SWEEP_BS) {
        const int k = row / n + 1, s = row - (k - 1) * n;
        double g = P.D[k][0] * z0[s];
        for (int j = 1; j <= KC; ++j) g += P.D[k][j] * Z[(j - 1) * n + s];
        double f = 0.0;
        for (int e = P.nu_ptr[s]; e < P.nu_ptr[s + 1]; ++e)
          f += P.nu_v[e] * kr[P.nu_r[e]] * mon[(k - 1) * r + P.nu_r[e]];
        g -= P.h * f;
        dZ[row] = g;
        Jm[(size_t)row * ldj + dim] = (float)g;
      }
      if (tid == 0) s_flag = 0;
      __syncthreads();
      // FP32 LU with partial pivoting of [J | G]
      for (int c = 0; c < dim; ++c) {
        if (warp == 0) {
          float best = -1.f;
          int bidx = dim;
          for (int rr = c + lane; rr < dim; rr += 32) {
            const float v = fabsf(Jm[(size_t)rr * ldj + c]);
            if (v > best) { best = v; bidx = rr; }
          }
          for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
            if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
          }
          if (lane == 0) {
            s_piv = bidx;
            if (!(best > 0.f) || !isfinite(best)) s_flag = 1;
          }
        }
        __syncthreads();
        if (s_flag) break;
        const int piv = s_piv;
        if (piv != c)
          for (int cc = c + tid; cc <= dim; cc += SWEEP_BS) {
            const float t0 = Jm[(size_t)c * ldj + cc];
            Jm[(size_t)c * ldj + cc] = Jm[(size_t)piv * ldj + cc];
            Jm[(size_t)piv * ldj + cc] = t0;
          }
        __syncthreads();
        if (tid == 0) s_inv = 1.f / Jm[(size_t)c * ldj + c];
        __syncthreads();
        const float inv = s_inv;
        const int w = dim - c;   // columns c+1..dim
        for (int idx = tid; idx < (dim - c - 1) * w; idx += SWEEP_BS) {
          const int rr = c + 1 + idx / w, cc = c + 1 + idx % w;
          Jm[(size_t)rr * ldj + cc] -= (Jm[(size_t)rr * ldj + c] * inv) * Jm[(size_t)c * ldj + cc];
        }
        __syncthreads();
      }
      if (s_flag) break;
      // back substitution U dZ = g (FP32), columns eliminated from the right
      for (int c = dim - 1; c >= 0; --c) {
        if (tid == 0) s_inv = Jm[(size_t)c * ldj + dim] / Jm[(size_t)c * ldj + c];
        __syncthreads();
        const float xc = s_inv;
        for (int rr = tid; rr < c; rr += SWEEP_BS) Jm[(size_t)rr * ldj + dim] -= Jm[(size_t)rr * ldj + c] * xc;
        if (tid == 0) dZ[c] = (double)xc;
        __syncthreads();
      }
      double mdz = 0.0, mz = 0.0, bad = 0.0;
      for (int t = tid; t < dim; t += SWEEP_BS) {
        Z[t] -= dZ[t];
        if (!isfinite(Z[t])) bad = 1.0;
        mdz = fmax(mdz, fabs(dZ[t]));
        mz = fmax(mz, fabs(Z[t]));
      }
      mdz = bmax<SWEEP_BS>(mdz, s_red);
      mz = bmax<SWEEP_BS>(mz, s_red);
      bad = bmax<SWEEP_BS>(bad, s_red);
      if (bad > 0) break;
      if (mdz <= 1e-12 * fmax(1.0, mz)) { ok = true; break; }
    }
    __syncthreads();
    if (!ok) {
      ++nfail;
      for (int t = tid; t < dim; t += SWEEP_BS) Z[t] = z0[t % n];
      __syncthreads();
    }
    double* xi = x + (size_t)i * NP * n;
    for (int s = tid; s < n; s += SWEEP_BS) xi[s] = z0[s];
    for (int t = tid; t < dim; t += SWEEP_BS) xi[n + t] = Z[t];
    __syncthreads();
    for (int s = tid; s < n; s += SWEEP_BS) z0[s] = Z[(KC - 1) * n + s];
    __syncthreads();
  }
  if (tid == 0) *fails = nfail;
}

// The same sweep for 3n <= 32 on one warp: lane l owns row l of the FP32
// Newton matrix in registers, so the LU with partial pivoting and the back
// substitution run on warp shuffles without block barriers.
constexpr int WSWEEP = 32;
__global__ void __launch_bounds__(32) k_forward_sweep_warp(DevProb P, double* __restrict__ x,
                                                           int* __restrict__ fails) {
  extern __shared__ double sm[];
  const int n = P.n, r = P.r, dim = KC * n;
  const int lane = threadIdx.x;
  const unsigned FULL = 0xffffffffu;
  double* kr = sm;                 // [r]
  double* mon = kr + r;            // [3][r]
  float* daf = reinterpret_cast<float*>(mon + KC * r);   // [3][r]
  float* dbf = daf + KC * r;                             // [3][r]
  float* rows = dbf + KC * r;                            // [32][33] staging
  double* z0 = reinterpret_cast<double*>(rows + WSWEEP * (WSWEEP + 1));  // [n]
  double* Z = z0 + n;              // [3n]
  const size_t nz = (size_t)P.N * NP * n;
  for (int j = lane; j < r; j += 32) {
    const int q = P.pidx[j];
    if (q < 0) kr[j] = P.kfix[j];
    else kr[j] = P.logscale ? exp10(x[nz + q]) : x[nz + q];
  }
  for (int s = lane; s < n; s += 32) z0[s] = P.x0[s];
  __syncwarp();
  const int rk = lane < dim ? lane / n + 1 : 1;
  const int rs = lane < dim ? lane - (rk - 1) * n : 0;
  int nfail = 0;
  for (int i = 0; i < P.N; ++i) {
    for (int t = lane; t < dim; t += 32) Z[t] = z0[t % n];
    __syncwarp();
    bool ok = false;
    for (int it = 0; it < SWEEP_MAXIT; ++it) {
      for (int idx = lane; idx < KC * r; idx += 32) {
        const int k = idx / r, j = idx - k * r;
        const int a = P.react[2 * j], b = P.react[2 * j + 1];
        const double za = Z[k * n + a];
        if (b < 0) { mon[idx] = za; daf[idx] = 1.f; dbf[idx] = 0.f; }
        else { const double zb = Z[k * n + b]; mon[idx] = za * zb; daf[idx] = (float)zb; dbf[idx] = (float)za; }
      }
      __syncwarp();
      float* myrow = rows + lane * (WSWEEP + 1);
      double g = 0.0;
      if (lane < dim) {
        for (int c = 0; c < WSWEEP; ++c) myrow[c] = 0.f;
        for (int j = 1; j <= KC; ++j) myrow[(j - 1) * n + rs] = (float)P.D[rk][j];
        g = P.D[rk][0] * z0[rs];
        for (int j = 1; j <= KC; ++j) g += P.D[rk][j] * Z[(j - 1) * n + rs];
        double f = 0.0;
        const float hf = (float)P.h;
        for (int e = P.nu_ptr[rs]; e < P.nu_ptr[rs + 1]; ++e) {
          const int rr = P.nu_r[e];
          const int mi = (rk - 1) * r + rr;
          const double nk = P.nu_v[e] * kr[rr];
          f += nk * mon[mi];
          const float nkf = (float)nk;
          const int a = P.react[2 * rr], b = P.react[2 * rr + 1];
          myrow[(rk - 1) * n + a] -= hf * nkf * daf[mi];
          if (b >= 0) myrow[(rk - 1) * n + b] -= hf * nkf * dbf[mi];
        }
        g -= P.h * f;
      } else {
        for (int c = 0; c < WSWEEP; ++c) myrow[c] = 0.f;
      }
      __syncwarp();
      float row[WSWEEP];
#pragma unroll
      for (int c = 0; c < WSWEEP; ++c) row[c] = myrow[c];
      float rhs = (float)g;
      bool singular = false;
#pragma unroll
      for (int c = 0; c < WSWEEP; ++c) {
        if (c < dim && !singular) {
          float v = (lane >= c && lane < dim) ? fabsf(row[c]) : -1.f;
          int idx = lane;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(FULL, v, o);
            const int oi = __shfl_xor_sync(FULL, idx, o);
            if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
          }
          if (!(v > 0.f) || !isfinite(v)) {
            singular = true;
          } else {
            if (idx != c) {
              const int src = lane == c ? idx : (lane == idx ? c : lane);
#pragma unroll
              for (int k = c; k < WSWEEP; ++k) row[k] = __shfl_sync(FULL, row[k], src);
              rhs = __shfl_sync(FULL, rhs, src);
            }
            const float pv = __shfl_sync(FULL, row[c], c);
            const float f = (lane > c && lane < dim) ? row[c] / pv : 0.f;
#pragma unroll
            for (int k = c + 1; k < WSWEEP; ++k) {
              const float pk = __shfl_sync(FULL, row[k], c);
              row[k] -= f * pk;
            }
            const float pr = __shfl_sync(FULL, rhs, c);
            rhs -= f * pr;
          }
        }
      }
      if (singular) break;
      float sol = 0.f;
#pragma unroll
      for (int c = WSWEEP - 1; c >= 0; --c) {
        if (c < dim) {
          const float xc = __shfl_sync(FULL, rhs / row[c], c);
          if (lane < c) rhs -= row[c] * xc;
          if (lane == c) sol = xc;
        }
      }
      double mdz = 0.0, mz = 0.0;
      bool fin = true;
      if (lane < dim) {
        const double d = (double)sol;
        Z[lane] -= d;
        fin = isfinite(Z[lane]);
        mdz = fabs(d);
        mz = fabs(Z[lane]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mdz = fmax(mdz, __shfl_xor_sync(FULL, mdz, o));
        mz = fmax(mz, __shfl_xor_sync(FULL, mz, o));
      }
      fin = __all_sync(FULL, fin);
      __syncwarp();
      if (!fin) break;
      if (mdz <= 1e-12 * fmax(1.0, mz)) { ok = true; break; }
    }
    if (!ok) {
      ++nfail;
      for (int t = lane; t < dim; t += 32) Z[t] = z0[t % n];
      __syncwarp();
    }
    double* xi = x + (size_t)i * NP * n;
    for (int s = lane; s < n; s += 32) xi[s] = z0[s];
    for (int t = lane; t < dim; t += 32) xi[n + t] = Z[t];
    __syncwarp();
    for (int s = lane; s < n; s += 32) z0[s] = Z[(KC - 1) * n + s];
    __syncwarp();
  }
  if (lane == 0) *fails = nfail;
}

size_t sweep_smem_bytes(const DevProb& P, bool jm_in_smem) {
  const size_t dim = KC * (size_t)P.n;
  size_t v = sizeof(double) * ((size_t)P.r * (1 + 3 * KC) + P.n + 2 * dim);
  if (jm_in_smem) v += sizeof(float) * dim * (dim + 1);
  return v;
}

cudaError_t launch_forward_sweep(collo_problem* pr) {
  const DevProb& P = pr->P;
  if (KC * P.n <= WSWEEP) {
    size_t sm = sizeof(double) * ((size_t)P.r * (1 + KC) + P.n + KC * (size_t)P.n) +
                sizeof(float) * ((size_t)2 * KC * P.r + WSWEEP * (WSWEEP + 1));
    sm = (sm + 15) & ~size_t(15);
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(k_forward_sweep_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    count_launch();
    k_forward_sweep_warp<<<1, 32, sm, pr->stream>>>(P, pr->x, pr->fails);
    return cudaGetLastError();
  }
  const bool insm = pr->sweep_work == nullptr;
  size_t sm = sweep_smem_bytes(pr->P, insm);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_forward_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  count_launch();
  k_forward_sweep<<<1, SWEEP_BS, sm, pr->stream>>>(pr->P, pr->x, pr->fails, pr->sweep_work);
  return cudaGetLastError();
}

// Parameter-space quantities for barrier parameter mu:
//   sigma_theta = zl/sl + zu/su (into sigma[nz..]); bar = mu/sl - mu/su;
//   zlmzu = zl - zu; out[0] = max(sl zl, su zu), out[1] = min(...),
//   out[2] = sum zl + sum zu, out[3] = sum log sl + sum log su.
__global__ void __launch_bounds__(IBS)
k_theta_prep(DevProb P, const double* __restrict__ x, const double* __restrict__ zl,
             const double* __restrict__ zu, double mu, double* __restrict__ sigma,
             double* __restrict__ bar, double* __restrict__ zlmzu, double* __restrict__ out) {
  __shared__ double sh[IBS];
  const size_t nz = (size_t)P.N * NP * P.n;
  double wmax = 0.0, wmin = 1e300, zs = 0.0, lg = 0.0;
  for (int q = threadIdx.x; q < P.p; q += IBS) {
    const double th = x[nz + q];
    const double sl = th - P.theta_lo[q], su = P.theta_hi[q] - th;
    sigma[nz + q] = zl[q] / sl + zu[q] / su;
    bar[q] = mu / sl - mu / su;
    zlmzu[q] = zl[q] - zu[q];
    wmax = fmax(wmax, fmax(sl * zl[q], su * zu[q]));
    wmin = fmin(wmin, fmin(sl * zl[q], su * zu[q]));
    zs += zl[q] + zu[q];
    lg += log(sl) + log(su);
  }
  wmax = bmax<IBS>(wmax, sh);
  wmin = bmin<IBS>(wmin, sh);
  zs = bsum<IBS>(zs, sh);
  lg = bsum<IBS>(lg, sh);
  if (threadIdx.x == 0) { out[0] = wmax; out[1] = wmin; out[2] = zs; out[3] = lg; }
}

// Bound-dual steps, fraction-to-boundary step sizes and the barrier part of
// grad(phi_mu)^T dx:  out[0] = alpha_max, out[1] = alpha_z, out[2] = gphi_theta.
__global__ void __launch_bounds__(IBS)
k_theta_step(DevProb P, const double* __restrict__ x, const double* __restrict__ dx,
             const double* __restrict__ zl, const double* __restrict__ zu, double mu, double tau,
             double* __restrict__ dz, double* __restrict__ out) {
  __shared__ double sh[IBS];
  const size_t nz = (size_t)P.N * NP * P.n;
  double amax = 1.0, az = 1.0, g = 0.0;
  for (int q = threadIdx.x; q < P.p; q += IBS) {
    const double th = x[nz + q], d = dx[nz + q];
    const double sl = th - P.theta_lo[q], su = P.theta_hi[q] - th;
    const double dzl = mu / sl - zl[q] - (zl[q] / sl) * d;
    const double dzu = mu / su - zu[q] + (zu[q] / su) * d;
    dz[q] = dzl;
    dz[P.p + q] = dzu;
    if (d < 0) amax = fmin(amax, -tau * sl / d);
    if (-d < 0) amax = fmin(amax, tau * su / d);
    if (dzl < 0) az = fmin(az, -tau * zl[q] / dzl);
    if (dzu < 0) az = fmin(az, -tau * zu[q] / dzu);
    g += (-mu / sl + mu / su) * d;
  }
  amax = bmin<IBS>(amax, sh);
  az = bmin<IBS>(az, sh);
  g = bsum<IBS>(g, sh);
  if (threadIdx.x == 0) { out[0] = amax; out[1] = az; out[2] = g; }
}

// Barrier log terms at the trial point theta + alpha dtheta.
// out[0] = sum log sl + log su, out[1] = 1 if all slacks > 0.
__global__ void __launch_bounds__(IBS)
k_trial_barrier(DevProb P, const double* __restrict__ x, const double* __restrict__ dx,
                double alpha, double* __restrict__ out) {
  __shared__ double sh[IBS];
  const size_t nz = (size_t)P.N * NP * P.n;
  double lg = 0.0, bad = 0.0;
  for (int q = threadIdx.x; q < P.p; q += IBS) {
    const double th = x[nz + q] + alpha * dx[nz + q];
    const double sl = th - P.theta_lo[q], su = P.theta_hi[q] - th;
    if (!(sl > 0) || !(su > 0)) bad = 1.0;
    else lg += log(sl) + log(su);
  }
  lg = bsum<IBS>(lg, sh);
  bad = bmax<IBS>(bad, sh);
  if (threadIdx.x == 0) { out[0] = lg; out[1] = bad > 0 ? 0.0 : 1.0; }
}

// Accept the step: x += alpha dx, lambda += alpha dlambda, bound duals
// += alpha_z dz, then reset into [mu/(kS s), kS mu/s].
__global__ void k_update(DevProb P, double* __restrict__ x, double* __restrict__ lam,
                         double* __restrict__ zl, double* __restrict__ zu,
                         const double* __restrict__ sol, const double* __restrict__ dz,
                         double alpha, double alpha_z, double mu, double ksig, size_t nx,
                         size_t nc) {
  const size_t nz = (size_t)P.N * NP * P.n;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (size_t i = tid; i < (size_t)P.p; i += stride) {
    const double th = x[nz + i] + alpha * sol[nz + i];
    const double sl = th - P.theta_lo[i], su = P.theta_hi[i] - th;
    double a = zl[i] + alpha_z * dz[i];
    double b = zu[i] + alpha_z * dz[P.p + i];
    a = fmax(fmin(a, ksig * mu / sl), mu / (ksig * sl));
    b = fmax(fmin(b, ksig * mu / su), mu / (ksig * su));
    zl[i] = a;
    zu[i] = b;
  }
  for (size_t i = tid; i < nx + nc; i += stride) {
    if (i < nx) x[i] += alpha * sol[i];
    else lam[i - nx] += alpha * sol[i];
  }
}

}  // namespace collo

using namespace collo;

namespace {

struct Opt {
  double tol, acc_tol;
  int acc_iter, max_iter;
  double max_wall;
  int precision;
  double mixed_mu_switch;
  int refine_max;
  double refine_tol;
  int verbose;
  // Waechter & Biegler (2006) constants
  double mu_init = 0.1, kappa_mu = 0.2, theta_mu = 1.5, kappa_eps = 10.0, tau_min = 0.99;
  double s_max = 100.0, kappa1 = 1e-2, kappa2 = 1e-2, kappa_sigma = 1e10;
  double gamma_theta = 1e-5, gamma_phi = 1e-5, delta = 1.0, s_theta = 1.1, s_phi = 2.3;
  double eta_phi = 1e-4, gamma_alpha = 0.05;
  double dw_min = 1e-20, dw_0 = 1e-4, dw_max = 1e40, kw_minus = 1.0 / 3.0, kw_plus = 8.0;
  double kw_plus_bar = 100.0, dc_coef = 1e-8, dc_exp = 0.25;
};

}  // namespace

extern "C" {

void collo_ipm_options_default(collo_ipm_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-6;
  o->acceptable_tol = 1e-4;
  o->acceptable_iter = 15;
  o->max_iter = 3000;
  o->max_wall_time = 3600.0;
  o->precision = COLLO_PRECISION_FP64;
  o->mixed_mu_switch = 1e-6;
  o->refine_max = 10;
  o->refine_tol = 1e-10;
  o->verbose = 0;
}

collo_status collo_initial_states(collo_problem* prob, const double* theta, double* x_out,
                                  int* failures) {
  if (!prob || !theta) { set_error("NULL argument"); return COLLO_ERR_INVALID_ARG; }
  COLLO_CUDA(cudaSetDevice(prob->device));
  cudaStream_t st = prob->stream;
  const size_t nz = (size_t)prob->P.N * NP * prob->P.n;
  if (prob->P.p)
    COLLO_CUDA(cudaMemcpyAsync(prob->x + nz, theta, prob->P.p * sizeof(double),
                               cudaMemcpyDefault, st));
  COLLO_CUDA(launch_forward_sweep(prob));
  int f = 0;
  COLLO_CUDA(cudaMemcpyAsync(&f, prob->fails, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (x_out)
    COLLO_CUDA(cudaMemcpyAsync(x_out, prob->x, prob->n_x * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  if (failures) *failures = f;
  return COLLO_OK;
}

collo_status collo_ipm_solve(collo_problem* prob, const double* theta0,
                             const collo_ipm_options* opts, collo_result* res) {
  if (!prob || !res || (prob->P.p > 0 && !theta0)) {
    set_error("NULL argument");
    return COLLO_ERR_INVALID_ARG;
  }
  COLLO_CUDA(cudaSetDevice(prob->device));
  collo_ipm_options uo;
  if (opts) uo = *opts; else collo_ipm_options_default(&uo);
  Opt o;
  o.tol = uo.tol; o.acc_tol = uo.acceptable_tol; o.acc_iter = uo.acceptable_iter;
  o.max_iter = uo.max_iter; o.max_wall = uo.max_wall_time; o.precision = uo.precision;
  o.mixed_mu_switch = uo.mixed_mu_switch; o.refine_max = uo.refine_max;
  o.refine_tol = uo.refine_tol; o.verbose = uo.verbose;
  const auto t_start = std::chrono::steady_clock::now();
  cudaStream_t st = prob->stream;
  const DevProb& P = prob->P;
  const int p = P.p;
  const size_t nx = prob->n_x, nc = prob->n_c, nz = nx - p;
  double* h = prob->hscal;
  double* d = prob->scal;
  double* bar = prob->thx;            // [p]
  double* zlmzu = prob->thx + p;      // [p]
  double* th0 = prob->thx + 2 * p;    // [p]
  double* dots = prob->red_parts;     // [RGRID] reduction partials
  double* rhs = prob->kvec_a;
  double* sol = prob->kvec_b;

  res->status = COLLO_ERR_MAXITER;
  res->iterations = 0; res->factorizations = 0; res->line_search_trials = 0;

  // initial point
  if (p) COLLO_CUDA(cudaMemcpyAsync(th0, theta0, p * sizeof(double), cudaMemcpyDefault, st));
  count_launch();
  k_init_point<<<1, 256, 0, st>>>(P, th0, prob->x, prob->zl, prob->zu, o.kappa1, o.kappa2);
  COLLO_CUDA(cudaGetLastError());
  COLLO_CUDA(launch_forward_sweep(prob));
  COLLO_CUDA(cudaMemsetAsync(prob->lam, 0, nc * sizeof(double), st));
  double mu = o.mu_init;
  double tau = std::max(o.tau_min, 1.0 - mu);
  std::vector<std::pair<double, double>> filt;
  double dw_last = 0.0;
  int acc_count = 0;
  COLLO_CUDA(launch_eval(P, prob->E, prob->x, nullptr, 0.0, nullptr, 1.0, false, st));
  COLLO_CUDA(cudaMemcpyAsync(h, prob->E.red, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  const double th_init = h[1];
  const double theta_max = 1e4 * std::max(1.0, th_init);
  const double theta_min = 1e-4 * std::max(1.0, th_init);
  int it = 0;
  double err = INFINITY, phi = NAN;
  collo_status status = COLLO_ERR_MAXITER;
  const long long want_pos = (long long)nx, want_neg = (long long)nc;

  for (;;) {
    double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    // 1. derivatives at the iterate and the optimality measures
    COLLO_CUDA(launch_eval(P, prob->E, prob->x, nullptr, 0.0, prob->lam, 1.0, true, st));
    prob->evaluated = true;
    count_launch();
    k_theta_prep<<<1, IBS, 0, st>>>(P, prob->x, prob->zl, prob->zu, mu, prob->sigma, bar, zlmzu,
                                    d + 16);
    COLLO_CUDA(launch_kkt_resid(P, prob->E, nullptr, 0.0, 0.0, nullptr, prob->lam,
                                prob->E.grad, -1.0, nullptr, 0.0, nullptr, prob->thpart,
                                prob->npart, zlmzu, d + 20, st));
    count_launch();
    k_dot_part<<<RGRID, IBS, 0, st>>>(prob->lam, nullptr, nc, 1, dots);
    count_launch();
    k_sum_parts<<<1, IBS, 0, st>>>(dots, d + 24);
    COLLO_CUDA(cudaGetLastError());
    COLLO_CUDA(cudaMemcpyAsync(h + 16, d + 16, 9 * sizeof(double), cudaMemcpyDeviceToHost, st));
    COLLO_CUDA(cudaMemcpyAsync(h, prob->E.red, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    COLLO_CUDA(cudaStreamSynchronize(st));
    phi = h[0];
    const double cinf = h[2];
    if (!std::isfinite(phi) || !std::isfinite(h[1])) { status = COLLO_ERR_NUMERIC; break; }
    const double wmax = h[16], wmin = h[17], zsum = h[18];
    const double dual = h[20], lam1 = h[24];
    const double s_d = std::max(o.s_max, (lam1 + zsum) / (double)(nc + 2 * p)) / o.s_max;
    const double s_c = std::max(o.s_max, zsum / (double)std::max(2 * p, 1)) / o.s_max;
    auto Emu = [&](double m) {
      double compl_ = p ? std::max(wmax - m, m - wmin) : 0.0;
      return std::max(std::max(dual / s_d, cinf), compl_ / s_c);
    };
    err = Emu(0.0);
    if (err <= o.tol) { status = COLLO_OK; break; }
    acc_count = err <= o.acc_tol ? acc_count + 1 : 0;
    if (acc_count >= o.acc_iter) { status = COLLO_ACCEPTABLE; break; }
    if (it >= o.max_iter) { status = COLLO_ERR_MAXITER; break; }
    if (wall > o.max_wall) { status = COLLO_ERR_TIMEOUT; break; }
    // 2. barrier update (monotone)
    while (Emu(mu) <= o.kappa_eps * mu) {
      double nm = std::max(o.tol / 10.0, std::min(o.kappa_mu * mu, std::pow(mu, o.theta_mu)));
      if (nm >= mu) break;
      mu = nm;
      tau = std::max(o.tau_min, 1.0 - mu);
      filt.clear();
    }
    // 3. Newton direction with inertia correction
    count_launch();
    k_theta_prep<<<1, IBS, 0, st>>>(P, prob->x, prob->zl, prob->zu, mu, prob->sigma, bar, zlmzu,
                                    d + 16);
    COLLO_CUDA(launch_kkt_resid(P, prob->E, nullptr, 0.0, 0.0, nullptr, prob->lam,
                                prob->E.grad, -1.0, prob->E.c, -1.0, rhs, prob->thpart,
                                prob->npart, bar, d + 20, st));
    const int prec = (o.precision == COLLO_PRECISION_MIXED &&
                      !(o.mixed_mu_switch > 0 && mu < o.mixed_mu_switch))
                         ? COLLO_PRECISION_MIXED : COLLO_PRECISION_FP64;
    const double dc = o.dc_coef * std::pow(mu, o.dc_exp);
    double dw = 0.0;
    long long in[3];
    collo_status s = factor_internal(prob, dw, dc, prec, in);
    if (s != COLLO_OK) return res->status = s;
    res->factorizations++;
    if (!(in[0] == want_pos && in[1] == want_neg && in[2] == 0)) {
      dw = dw_last == 0.0 ? o.dw_0 : std::max(o.dw_min, o.kw_minus * dw_last);
      bool good = false;
      for (;;) {
        s = factor_internal(prob, dw, dc, prec, in);
        if (s != COLLO_OK) return res->status = s;
        res->factorizations++;
        if (in[0] == want_pos && in[1] == want_neg && in[2] == 0) { good = true; dw_last = dw; break; }
        dw *= dw_last == 0.0 ? o.kw_plus_bar : o.kw_plus;
        if (dw > o.dw_max) break;
      }
      if (!good) { status = COLLO_ERR_INERTIA; break; }
    }
    int sweeps = 0;
    double rres = 0.0;
    s = solve_internal(prob, rhs, sol, o.refine_max, o.refine_tol, &sweeps, &rres);
    if (s != COLLO_OK) { status = s; break; }
    // 4. step sizes
    count_launch();
    k_theta_step<<<1, IBS, 0, st>>>(P, prob->x, sol, prob->zl, prob->zu, mu, tau, prob->dz, d + 28);
    count_launch();
    k_dot_part<<<RGRID, IBS, 0, st>>>(prob->E.grad, sol, nx, 0, dots);
    count_launch();
    k_sum_parts<<<1, IBS, 0, st>>>(dots, d + 32);
    COLLO_CUDA(cudaGetLastError());
    COLLO_CUDA(cudaMemcpyAsync(h + 16, d + 16, 17 * sizeof(double), cudaMemcpyDeviceToHost, st));
    COLLO_CUDA(cudaStreamSynchronize(st));
    const double alpha_max = h[28], alpha_z = h[29];
    const double gphi = h[32] + h[30];
    const double theta_k = h[1] > 0 ? h[1] : 0.0;
    const double phi_k = phi - mu * h[19];
    double alpha_min;
    if (gphi < 0) {
      if (theta_k <= theta_min)
        alpha_min = o.gamma_alpha * std::min(std::min(o.gamma_theta, o.gamma_phi * theta_k / (-gphi)),
                                             o.delta * std::pow(theta_k, o.s_theta) /
                                                 std::pow(-gphi, o.s_phi));
      else
        alpha_min = o.gamma_alpha * std::min(o.gamma_theta, o.gamma_phi * theta_k / (-gphi));
    } else {
      alpha_min = o.gamma_alpha * o.gamma_theta;
    }
    // 5. backtracking filter line search
    double alpha = alpha_max;
    bool accepted = false, ftype = false;
    int trials = 0;
    while (alpha >= alpha_min) {
      ++trials;
      COLLO_CUDA(launch_eval(P, prob->E, prob->x, sol, alpha, nullptr, 1.0, false, st));
      count_launch();
      k_trial_barrier<<<1, IBS, 0, st>>>(P, prob->x, sol, alpha, d + 36);
      COLLO_CUDA(cudaGetLastError());
      COLLO_CUDA(cudaMemcpyAsync(h, prob->E.red, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
      COLLO_CUDA(cudaMemcpyAsync(h + 36, d + 36, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      COLLO_CUDA(cudaStreamSynchronize(st));
      const double phit = h[0], thetat = h[1];
      if (std::isfinite(phit) && std::isfinite(thetat) && h[37] > 0.5) {
        const double phibt = phit - mu * h[36];
        bool ok = std::isfinite(phibt) && thetat < theta_max;
        if (ok)
          for (auto& f : filt)
            if (thetat >= f.first && phibt >= f.second) { ok = false; break; }
        if (ok) {
          const bool sw = gphi < 0 &&
                          alpha * std::pow(-gphi, o.s_phi) > o.delta * std::pow(theta_k, o.s_theta);
          if (theta_k <= theta_min && sw) {
            ftype = true;
            accepted = phibt <= phi_k + o.eta_phi * alpha * gphi;
          } else {
            ftype = false;
            accepted = thetat <= (1.0 - o.gamma_theta) * theta_k || phibt <= phi_k - o.gamma_phi * theta_k;
          }
          if (accepted) break;
        }
      }
      alpha *= 0.5;
    }
    res->line_search_trials += trials;
    if (!accepted) { status = COLLO_ERR_LINESEARCH; break; }
    if (!ftype) filt.push_back({(1.0 - o.gamma_theta) * theta_k, phi_k - o.gamma_phi * theta_k});
    count_launch();
    k_update<<<std::min<size_t>((nx + nc + 255) / 256, 8192), 256, 0, st>>>(
        P, prob->x, prob->lam, prob->zl, prob->zu, sol, prob->dz, alpha, alpha_z, mu,
        o.kappa_sigma, nx, nc);
    COLLO_CUDA(cudaGetLastError());
    if (o.verbose)
      std::printf("iter %4d phi %.10e inf_pr %.3e err %.3e mu %.3e dw %.2e alpha %.3e ls %d ir %d %s\n",
                  it, phi, cinf, err, mu, dw, alpha, trials, sweeps,
                  prec == COLLO_PRECISION_MIXED ? "fp32+ir" : "fp64");
    ++it;
  }
  res->status = status;
  res->iterations = it;
  res->phi = phi;
  res->kkt_error = err;
  res->mu = mu;
  if (res->theta && p)
    COLLO_CUDA(cudaMemcpyAsync(res->theta, prob->x + nz, p * sizeof(double), cudaMemcpyDefault, st));
  if (res->x)
    COLLO_CUDA(cudaMemcpyAsync(res->x, prob->x, nx * sizeof(double), cudaMemcpyDefault, st));
  if (res->lambda)
    COLLO_CUDA(cudaMemcpyAsync(res->lambda, prob->lam, nc * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  res->wall_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  return status;
}

}  // extern "C"
