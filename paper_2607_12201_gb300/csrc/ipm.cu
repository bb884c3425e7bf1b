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
  const size_t nz = (size_t)P.N * P.np * P.n;
  for (int q = threadIdx.x; q < P.p; q += blockDim.x) {
    const double lo = P.theta_lo[q], hi = P.theta_hi[q];
    const double pl = fmin(kappa1 * fmax(1.0, fabs(lo)), kappa2 * (hi - lo));
    const double pu = fmin(kappa1 * fmax(1.0, fabs(hi)), kappa2 * (hi - lo));
    x[nz + q] = fmin(fmax(theta0[q], lo + pl), hi - pu);
    zl[q] = 1.0;
    zu[q] = 1.0;
  }
}

// State at the element's end, the next element's z0 (Eq. 2c): Radau z_K
// (tau_K = 1); Gauss the extrapolation sum_j b_j z_j, j = 0..K, with z_0 = z0
// and z_j = Z[j - 1] (same order of terms as the continuity residual).
__device__ inline double end_state(const DevProb& P, const double* z0, const double* Z, int s) {
  const int n = P.n;
  if (!P.gauss) return Z[(P.K - 1) * n + s];
  double v = P.bw[0] * z0[s];
  for (int j = 1; j <= P.K; ++j) v += P.bw[j] * Z[(j - 1) * n + s];
  return v;
}

// Collocation forward sweep at theta = x[nz..]: for each element in turn,
// Newton's method on the K collocation equations in the element's interior
// states, started at the element's initial state, stopped when
// max|dZ| <= 1e-12 max(1, max|Z|) (at most 30 iterations); an element whose
// iteration fails keeps the constant guess.  The residual, the update and
// the stopping test are FP64; the Newton correction solves the Jacobian
// system by an FP32 LU with partial pivoting (an inexact Newton step whose
// error the FP64 residual of the next iteration corrects), so the sweep
// converges to the same FP64 collocation solution.  One block of SWEEP_BS
// threads.  The LU carries the residual as an extra column (so the forward
// substitution happens during the elimination) and runs with two barriers
// per column: warp 0 picks the pivot among a compact list of the rows not yet
// pivoted (rows are exchanged only in that list), then the block updates
// those rows, one warp per row and the lanes along the columns.  The back
// substitution runs on warp 0.  The FP32 matrix [J | G] sits in shared
// memory, or in gwork when Kn is too large.
constexpr int SWEEP_MAXIT = 30;
constexpr int SWEEP_BS = 1024;

// Maxima of three values over a block of BS threads: shuffle trees within the
// warps, then over the warps' maxima; two barriers.  sh: 3 (BS / 32 + 1) doubles.
template <int BS>
__device__ void bmax3(double& a, double& b, double& c, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = BS / 32;
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    c = fmax(c, __shfl_xor_sync(0xffffffffu, c, o));
  }
  if (lane == 0) { sh[3 * warp] = a; sh[3 * warp + 1] = b; sh[3 * warp + 2] = c; }
  __syncthreads();
  if (warp == 0) {
    a = lane < NW ? sh[3 * lane] : 0.0;
    b = lane < NW ? sh[3 * lane + 1] : 0.0;
    c = lane < NW ? sh[3 * lane + 2] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
      c = fmax(c, __shfl_xor_sync(0xffffffffu, c, o));
    }
    if (lane == 0) { sh[3 * NW] = a; sh[3 * NW + 1] = b; sh[3 * NW + 2] = c; }
  }
  __syncthreads();
  a = sh[3 * NW]; b = sh[3 * NW + 1]; c = sh[3 * NW + 2];
}

// Bytes of sweep_cta's dynamic shared memory before the matrix.
__host__ __device__ inline size_t sweep_cta_vec_bytes(const DevProb& P) {
  const size_t dim = P.K * (size_t)P.n;
  return sizeof(double) * ((size_t)P.r * (1 + 3 * P.K) + P.n + 2 * dim) +
         sizeof(float) * dim + sizeof(int) * 2 * dim;
}

__device__ void sweep_cta(const DevProb& P, double* __restrict__ x, int* __restrict__ fails,
                          float* __restrict__ gwork, double* sm) {
  __shared__ double s_red[3 * (SWEEP_BS / 32 + 1)];
  __shared__ int s_flag;
  const int n = P.n, r = P.r, K = P.K, dim = K * n, ldj = dim + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* kr = sm;                 // [r]
  double* mon = kr + r;            // [K][r]
  double* da = mon + K * r;        // [K][r]
  double* db = da + K * r;         // [K][r]
  double* z0 = db + K * r;         // [n]
  double* Z = z0 + n;              // [Kn]
  double* dZ = Z + dim;            // [Kn]  Newton correction
  float* inv = reinterpret_cast<float*>(dZ + dim);    // [Kn]  1 / U[c][c]
  int* perm = reinterpret_cast<int*>(inv + dim);      // [Kn]  row pivoted at step c
  int* rem = perm + dim;           // [Kn]  rows not yet pivoted (first dim - c)
  float* Jm = gwork ? gwork : reinterpret_cast<float*>(rem + dim);  // [dim][dim+1]
  const size_t nz = (size_t)P.N * P.np * n;
  int nfail = 0;
  for (int i = 0; i < P.N; ++i) {
    if (chain_start(P, i)) {   // a condition's first element: its rates and x0
      const int c = i / P.Nch;
      for (int j = tid; j < r; j += SWEEP_BS) {
        const int q = P.pidx[j];
        double k = q < 0 ? P.kfix[j] : (P.logscale ? exp10(x[nz + q]) : x[nz + q]);
        if (P.kscale) k *= P.kscale[(size_t)c * r + j];
        kr[j] = k;
      }
      for (int s = tid; s < n; s += SWEEP_BS) z0[s] = P.x0[(size_t)c * n + s];
      __syncthreads();
    }
    for (int t = tid; t < dim; t += SWEEP_BS) Z[t] = z0[t % n];
    __syncthreads();
    bool ok = false;
    for (int it = 0; it < SWEEP_MAXIT; ++it) {
      for (int idx = tid; idx < K * r; idx += SWEEP_BS) {
        const int k = idx / r, j = idx - k * r;
        const int a = P.react[2 * j], b = P.react[2 * j + 1];
        const double za = Z[k * n + a];
        if (b < 0) { mon[idx] = za; da[idx] = 1.0; db[idx] = 0.0; }
        else { const double zb = Z[k * n + b]; mon[idx] = za * zb; da[idx] = zb; db[idx] = za; }
      }
      __syncthreads();
      // Jacobian entries D[k][j] delta_st - delta_kj h df_s/dz_t (FP32) and the
      // residual G (FP64, rounded to FP32 in column dim)
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
        for (int j = 1; j <= K; ++j) g += P.D[k][j] * Z[(j - 1) * n + s];
        double f = 0.0;
        for (int e = P.nu_ptr[s]; e < P.nu_ptr[s + 1]; ++e)
          f += P.nu_v[e] * kr[P.nu_r[e]] * mon[(k - 1) * r + P.nu_r[e]];
        g -= P.h * f;
        Jm[(size_t)row * ldj + dim] = (float)g;
        rem[row] = row;
      }
      if (tid == 0) s_flag = 0;
      __syncthreads();
      // FP32 LU with partial pivoting of [J | G]; L[r][c] = Jm[r][c] inv[c]
      // (column c of a row is not updated after step c)
      for (int c = 0; c < dim; ++c) {
        const int nrem = dim - c;
        if (warp == 0) {
          float best = -1.f;
          int bpos = nrem, brow = dim;
          for (int q = lane; q < nrem; q += 32) {
            const int rr = rem[q];
            const float v = fabsf(Jm[(size_t)rr * ldj + c]);
            if (v > best || (v == best && rr < brow)) { best = v; bpos = q; brow = rr; }
          }
          for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int op = __shfl_xor_sync(0xffffffffu, bpos, o);
            const int orow = __shfl_xor_sync(0xffffffffu, brow, o);
            if (ob > best || (ob == best && orow < brow)) { best = ob; bpos = op; brow = orow; }
          }
          if (lane == 0) {
            if (!(best > 0.f) || !isfinite(best)) {
              s_flag = 1;
            } else {
              perm[c] = brow;
              inv[c] = 1.f / Jm[(size_t)brow * ldj + c];
              rem[bpos] = rem[nrem - 1];   // the pivot row leaves the list
            }
          }
        }
        __syncthreads();
        if (s_flag) break;
        const int piv = perm[c];
        const float ic = inv[c];
        const float* prow = Jm + (size_t)piv * ldj;
        for (int q = warp; q < nrem - 1; q += SWEEP_BS / 32) {
          float* row = Jm + (size_t)rem[q] * ldj;
          const float m = row[c] * ic;
          for (int cc = c + 1 + lane; cc <= dim; cc += 32) row[cc] -= m * prow[cc];
        }
        __syncthreads();
      }
      if (s_flag) break;
      // back substitution U dZ = y on warp 0 (U row c is row perm[c])
      if (warp == 0) {
        for (int c = dim - 1; c >= 0; --c) {
          const float xc = Jm[(size_t)perm[c] * ldj + dim] * inv[c];
          for (int q = lane; q < c; q += 32) {
            float* row = Jm + (size_t)perm[q] * ldj;
            row[dim] -= row[c] * xc;
          }
          if (lane == 0) dZ[c] = (double)xc;
          __syncwarp();
        }
      }
      __syncthreads();
      double mdz = 0.0, mz = 0.0, bad = 0.0;
      for (int t = tid; t < dim; t += SWEEP_BS) {
        Z[t] -= dZ[t];
        if (!isfinite(Z[t])) bad = 1.0;
        mdz = fmax(mdz, fabs(dZ[t]));
        mz = fmax(mz, fabs(Z[t]));
      }
      bmax3<SWEEP_BS>(mdz, mz, bad, s_red);
      if (bad > 0) break;
      if (mdz <= 1e-12 * fmax(1.0, mz)) { ok = true; break; }
    }
    __syncthreads();
    if (!ok) {
      ++nfail;
      for (int t = tid; t < dim; t += SWEEP_BS) Z[t] = z0[t % n];
      __syncthreads();
    }
    double* xi = x + (size_t)i * P.np * n;
    for (int s = tid; s < n; s += SWEEP_BS) xi[s] = z0[s];
    for (int t = tid; t < dim; t += SWEEP_BS) xi[n + t] = Z[t];
    __syncthreads();
    for (int s = tid; s < n; s += SWEEP_BS) z0[s] = end_state(P, z0, Z, s);
    __syncthreads();
  }
  if (tid == 0) *fails = nfail;
}

__global__ void __launch_bounds__(SWEEP_BS) k_forward_sweep(DevProb P, double* __restrict__ x,
                                                            int* __restrict__ fails,
                                                            float* __restrict__ gwork) {
  extern __shared__ double sm[];
  sweep_cta(P, x, fails, gwork, sm);
}

// The same sweep for Kn <= 32 on one warp: lane l owns row l of the FP32
// Newton matrix in registers, so the LU with partial pivoting and the
// substitutions run on warp shuffles without block barriers.  The Newton
// iteration is a chord iteration: the LU's multipliers (lrow, per step and
// lane, as they were applied) and pivot rows are kept, later iterations
// replay the same elimination on the new residual, and the matrix is
// refactored only when the step shrinks by less than CHORD_RATE.  Each
// element starts from the previous element's stage increments added to its
// initial state.
constexpr int WSWEEP = 32;
constexpr double CHORD_RATE = 0.25;
__device__ void sweep_warp(const DevProb& P, double* __restrict__ x, int* __restrict__ fails,
                           double* sm) {
  const int n = P.n, r = P.r, K = P.K, dim = K * n;
  const int lane = threadIdx.x;
  const unsigned FULL = 0xffffffffu;
  double* kr = sm;                 // [r]
  double* mon = kr + r;            // [K][r]
  float* daf = reinterpret_cast<float*>(mon + K * r);   // [K][r]
  float* dbf = daf + K * r;                             // [K][r]
  float* rows = dbf + K * r;                            // [32][33] staging
  double* z0 = reinterpret_cast<double*>(rows + WSWEEP * (WSWEEP + 1));  // [n]
  double* Z = z0 + n;              // [Kn]
  const size_t nz = (size_t)P.N * P.np * n;
  const int rk = lane < dim ? lane / n + 1 : 1;
  const int rs = lane < dim ? lane - (rk - 1) * n : 0;
  int nfail = 0;
  float row[WSWEEP], lrow[WSWEEP];
  int piv[WSWEEP];
  double dZ = 0.0;                 // lane's stage increment in the previous element
  for (int i = 0; i < P.N; ++i) {
    if (chain_start(P, i)) {   // a condition's first element: its rates and x0
      const int c = i / P.Nch;
      for (int j = lane; j < r; j += 32) {
        const int q = P.pidx[j];
        double k = q < 0 ? P.kfix[j] : (P.logscale ? exp10(x[nz + q]) : x[nz + q]);
        if (P.kscale) k *= P.kscale[(size_t)c * r + j];
        kr[j] = k;
      }
      for (int s = lane; s < n; s += 32) z0[s] = P.x0[(size_t)c * n + s];
      dZ = 0.0;
      __syncwarp();
    }
    if (lane < dim) Z[lane] = z0[rs] + dZ;
    __syncwarp();
    bool ok = false, have_lu = false;
    double mdz_prev = 0.0;
    for (int it = 0; it < SWEEP_MAXIT; ++it) {
      const bool refactor = !have_lu;
      for (int idx = lane; idx < K * r; idx += 32) {
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
        if (refactor) {
          for (int c = 0; c < WSWEEP; ++c) myrow[c] = 0.f;
          for (int j = 1; j <= K; ++j) myrow[(j - 1) * n + rs] = (float)P.D[rk][j];
        }
        g = P.D[rk][0] * z0[rs];
        for (int j = 1; j <= K; ++j) g += P.D[rk][j] * Z[(j - 1) * n + rs];
        double f = 0.0;
        const float hf = (float)P.h;
        for (int e = P.nu_ptr[rs]; e < P.nu_ptr[rs + 1]; ++e) {
          const int rr = P.nu_r[e];
          const int mi = (rk - 1) * r + rr;
          const double nk = P.nu_v[e] * kr[rr];
          f += nk * mon[mi];
          if (refactor) {
            const float nkf = (float)nk;
            const int a = P.react[2 * rr], b = P.react[2 * rr + 1];
            myrow[(rk - 1) * n + a] -= hf * nkf * daf[mi];
            if (b >= 0) myrow[(rk - 1) * n + b] -= hf * nkf * dbf[mi];
          }
        }
        g -= P.h * f;
      } else if (refactor) {
        for (int c = 0; c < WSWEEP; ++c) myrow[c] = 0.f;
      }
      __syncwarp();
      float rhs = (float)g;
      bool singular = false;
      if (refactor) {
#pragma unroll
        for (int c = 0; c < WSWEEP; ++c) row[c] = myrow[c];
#pragma unroll
        for (int c = 0; c < WSWEEP; ++c) {
          lrow[c] = 0.f;
          piv[c] = c;
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
              piv[c] = idx;
              if (idx != c) {
                const int src = lane == c ? idx : (lane == idx ? c : lane);
#pragma unroll
                for (int k = c; k < WSWEEP; ++k) row[k] = __shfl_sync(FULL, row[k], src);
                rhs = __shfl_sync(FULL, rhs, src);
              }
              const float pv = __shfl_sync(FULL, row[c], c);
              const float f = (lane > c && lane < dim) ? row[c] / pv : 0.f;
              lrow[c] = f;
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
        have_lu = true;
      } else {
        // replay the factorization's row exchanges and eliminations on rhs
#pragma unroll
        for (int c = 0; c < WSWEEP; ++c) {
          if (c < dim) {
            const int pc = piv[c];
            if (pc != c) {
              const int src = lane == c ? pc : (lane == pc ? c : lane);
              rhs = __shfl_sync(FULL, rhs, src);
            }
            const float pr = __shfl_sync(FULL, rhs, c);
            rhs -= lrow[c] * pr;
          }
        }
      }
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
      // slow contraction of the chord iteration: refactor at the current point
      if (it > 0 && mdz > CHORD_RATE * mdz_prev) have_lu = false;
      mdz_prev = mdz;
    }
    if (!ok) {
      ++nfail;
      for (int t = lane; t < dim; t += 32) Z[t] = z0[t % n];
      __syncwarp();
    }
    dZ = lane < dim ? Z[lane] - z0[rs] : 0.0;
    double* xi = x + (size_t)i * P.np * n;
    for (int s = lane; s < n; s += 32) xi[s] = z0[s];
    for (int t = lane; t < dim; t += 32) xi[n + t] = Z[t];
    __syncwarp();
    for (int s = lane; s < n; s += 32) z0[s] = end_state(P, z0, Z, s);
    __syncwarp();
  }
  if (lane == 0) *fails = nfail;
}

__global__ void __launch_bounds__(32) k_forward_sweep_warp(DevProb P, double* __restrict__ x,
                                                           int* __restrict__ fails) {
  extern __shared__ double sm[];
  sweep_warp(P, x, fails, sm);
}

size_t sweep_warp_smem_bytes(const DevProb& P) {
  size_t sm = sizeof(double) * ((size_t)P.r * (1 + P.K) + P.n + P.K * (size_t)P.n) +
              sizeof(float) * ((size_t)2 * P.K * P.r + WSWEEP * (WSWEEP + 1));
  return (sm + 15) & ~size_t(15);
}

// Batched sweeps: one block per instance.
__global__ void __launch_bounds__(32) k_sweep_warp_b(const DevInst* __restrict__ insts,
                                                     const int* __restrict__ act) {
  extern __shared__ double sm[];
  const DevInst& I = insts[act[blockIdx.x]];
  sweep_warp(I.P, I.x, I.fails, sm);
}
__global__ void __launch_bounds__(SWEEP_BS) k_sweep_cta_b(const DevInst* __restrict__ insts,
                                                          const int* __restrict__ act) {
  extern __shared__ double sm[];
  const DevInst& I = insts[act[blockIdx.x]];
  sweep_cta(I.P, I.x, I.fails, I.sweep_work, sm);
}

size_t sweep_smem_bytes(const DevProb& P, bool jm_in_smem) {
  const size_t dim = P.K * (size_t)P.n;
  size_t v = sweep_cta_vec_bytes(P);
  if (jm_in_smem) v += sizeof(float) * dim * (dim + 1);
  return v;
}

cudaError_t launch_forward_sweep(collo_problem* pr) {
  const DevProb& P = pr->P;
  if (P.K * P.n <= WSWEEP) {
    size_t sm = sweep_warp_smem_bytes(P);
    if (sm > SMEM_OPTIN_ABOVE)
      cudaFuncSetAttribute(k_forward_sweep_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    count_launch();
    k_forward_sweep_warp<<<1, 32, sm, pr->stream>>>(P, pr->x, pr->fails);
    return cudaGetLastError();
  }
  const bool insm = pr->sweep_work == nullptr;
  size_t sm = sweep_smem_bytes(pr->P, insm);
  if (sm > SMEM_OPTIN_ABOVE)
    cudaFuncSetAttribute(k_forward_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  count_launch();
  k_forward_sweep<<<1, SWEEP_BS, sm, pr->stream>>>(pr->P, pr->x, pr->fails, pr->sweep_work);
  return cudaGetLastError();
}

// ---- batched IPM kernels (one block per instance unless stated) ------------------

// theta0 pushed into the bounds (Waechter & Biegler 2006, Sec. 3.6), bound
// duals 1.
__global__ void k_init_point_b(const DevInst* __restrict__ insts, const int* __restrict__ act,
                               double kappa1, double kappa2) {
  const DevInst& I = insts[act[blockIdx.x]];
  const DevProb& P = I.P;
  const size_t nz = (size_t)P.N * P.np * P.n;
  for (int q = threadIdx.x; q < P.p; q += blockDim.x) {
    const double lo = P.theta_lo[q], hi = P.theta_hi[q];
    const double pl = fmin(kappa1 * fmax(1.0, fabs(lo)), kappa2 * (hi - lo));
    const double pu = fmin(kappa1 * fmax(1.0, fabs(hi)), kappa2 * (hi - lo));
    I.x[nz + q] = fmin(fmax(I.th0[q], lo + pl), hi - pu);
    I.zl[q] = 1.0;
    I.zu[q] = 1.0;
  }
}

// Parameter-space quantities for barrier parameter mu:
//   sigma_theta = zl/sl + zu/su (into sigma[nz..]); bar = mu/sl - mu/su;
//   zlmzu = zl - zu; out: max / min of (sl zl, su zu), sum zl + zu,
//   sum log sl + log su.
__global__ void __launch_bounds__(IBS)
k_theta_prep_b(const DevInst* __restrict__ insts, const int* __restrict__ act,
               const InstParams* __restrict__ prm) {
  __shared__ double sh[IBS];
  const DevInst& I = insts[act[blockIdx.x]];
  const DevProb& P = I.P;
  const double mu = prm[blockIdx.x].mu;
  const size_t nz = (size_t)P.N * P.np * P.n;
  double wmax = 0.0, wmin = 1e300, zs = 0.0, lg = 0.0;
  for (int q = threadIdx.x; q < P.p; q += IBS) {
    const double th = I.x[nz + q];
    const double sl = th - P.theta_lo[q], su = P.theta_hi[q] - th;
    I.sigma[nz + q] = I.zl[q] / sl + I.zu[q] / su;
    I.bar[q] = mu / sl - mu / su;
    I.zlmzu[q] = I.zl[q] - I.zu[q];
    wmax = fmax(wmax, fmax(sl * I.zl[q], su * I.zu[q]));
    wmin = fmin(wmin, fmin(sl * I.zl[q], su * I.zu[q]));
    zs += I.zl[q] + I.zu[q];
    lg += log(sl) + log(su);
  }
  wmax = bmax<IBS>(wmax, sh);
  wmin = bmin<IBS>(wmin, sh);
  zs = bsum<IBS>(zs, sh);
  lg = bsum<IBS>(lg, sh);
  if (threadIdx.x == 0) {
    I.out[O_WMAX] = wmax; I.out[O_WMIN] = wmin; I.out[O_ZSUM] = zs; I.out[O_LOG] = lg;
  }
}

// |lambda|_1 (which = 0) or grad^T kb over the primal entries (which = 1).
__global__ void __launch_bounds__(IBS)
k_vec_reduce_b(const DevInst* __restrict__ insts, const int* __restrict__ act, int which) {
  __shared__ double sh[IBS];
  const DevInst& I = insts[act[blockIdx.x]];
  double v = 0.0;
  if (which == 0)
    for (long long i = threadIdx.x; i < I.n_c; i += IBS) v += fabs(I.lam[i]);
  else
    for (long long i = threadIdx.x; i < I.n_x; i += IBS) v += I.E.grad[i] * I.kb[i];
  v = bsum<IBS>(v, sh);
  if (threadIdx.x == 0) I.out[which == 0 ? O_LAM1 : O_GDX] = v;
}

// Bound-dual steps, fraction-to-boundary step sizes and the barrier part of
// grad(phi_mu)^T dx.
__global__ void __launch_bounds__(IBS)
k_theta_step_b(const DevInst* __restrict__ insts, const int* __restrict__ act,
               const InstParams* __restrict__ prm) {
  __shared__ double sh[IBS];
  const DevInst& I = insts[act[blockIdx.x]];
  const DevProb& P = I.P;
  const double mu = prm[blockIdx.x].mu, tau = prm[blockIdx.x].tau;
  const size_t nz = (size_t)P.N * P.np * P.n;
  double amax = 1.0, az = 1.0, g = 0.0;
  for (int q = threadIdx.x; q < P.p; q += IBS) {
    const double th = I.x[nz + q], d = I.kb[nz + q];
    const double sl = th - P.theta_lo[q], su = P.theta_hi[q] - th;
    const double dzl = mu / sl - I.zl[q] - (I.zl[q] / sl) * d;
    const double dzu = mu / su - I.zu[q] + (I.zu[q] / su) * d;
    I.dz[q] = dzl;
    I.dz[P.p + q] = dzu;
    if (d < 0) amax = fmin(amax, -tau * sl / d);
    if (-d < 0) amax = fmin(amax, tau * su / d);
    if (dzl < 0) az = fmin(az, -tau * I.zl[q] / dzl);
    if (dzu < 0) az = fmin(az, -tau * I.zu[q] / dzu);
    g += (-mu / sl + mu / su) * d;
  }
  amax = bmin<IBS>(amax, sh);
  az = bmin<IBS>(az, sh);
  g = bsum<IBS>(g, sh);
  if (threadIdx.x == 0) { I.out[O_AMAX] = amax; I.out[O_AZ] = az; I.out[O_GPHI] = g; }
}

// Barrier log terms at the trial point theta + alpha dtheta.
__global__ void __launch_bounds__(IBS)
k_trial_barrier_b(const DevInst* __restrict__ insts, const int* __restrict__ act,
                  const InstParams* __restrict__ prm) {
  __shared__ double sh[IBS];
  const DevInst& I = insts[act[blockIdx.x]];
  const DevProb& P = I.P;
  const double alpha = prm[blockIdx.x].alpha;
  const size_t nz = (size_t)P.N * P.np * P.n;
  double lg = 0.0, bad = 0.0;
  for (int q = threadIdx.x; q < P.p; q += IBS) {
    const double th = I.x[nz + q] + alpha * I.kb[nz + q];
    const double sl = th - P.theta_lo[q], su = P.theta_hi[q] - th;
    if (!(sl > 0) || !(su > 0)) bad = 1.0;
    else lg += log(sl) + log(su);
  }
  lg = bsum<IBS>(lg, sh);
  bad = bmax<IBS>(bad, sh);
  if (threadIdx.x == 0) { I.out[O_TLOG] = lg; I.out[O_TOK] = bad > 0 ? 0.0 : 1.0; }
}

// Grid-stride over the n_x + n_c entries of every active instance (prefix
// pre): mode 0 accepts the step (x += alpha dx, lambda += alpha dlambda,
// bound duals += alpha_z dz then reset into [mu/(kS s), kS mu/s]); mode 1
// adds the refinement correction (kb += kc); mode 2 zeroes lambda.
__global__ void k_update_b(const DevInst* __restrict__ insts, const int* __restrict__ act, int A,
                           const long long* __restrict__ pre, const InstParams* __restrict__ prm,
                           int mode) {
  const long long total = pre[A];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = A;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pre[mid] <= t) lo = mid; else hi = mid;
    }
    const int k = lo;
    const DevInst& I = insts[act[k]];
    const long long j = t - pre[k];
    if (mode == 1) { I.kb[j] += I.kc[j]; continue; }
    if (mode == 2) { if (j < I.n_c) I.lam[j] = 0.0; continue; }
    const InstParams pr = prm[k];
    const long long nz = I.n_x - I.P.p;
    if (j >= nz && j < I.n_x) {
      // parameter entry q: the same thread moves theta_q and its bound duals
      const DevProb& P = I.P;
      const int q = (int)(j - nz);
      const double th = I.x[j] + pr.alpha * I.kb[j];
      I.x[j] = th;
      const double sl = th - P.theta_lo[q], su = P.theta_hi[q] - th;
      double a = I.zl[q] + pr.alpha_z * I.dz[q];
      double b = I.zu[q] + pr.alpha_z * I.dz[P.p + q];
      a = fmax(fmin(a, pr.ksig * pr.mu / sl), pr.mu / (pr.ksig * sl));
      b = fmax(fmin(b, pr.ksig * pr.mu / su), pr.mu / (pr.ksig * su));
      I.zl[q] = a;
      I.zu[q] = b;
    } else if (j < I.n_x) {
      I.x[j] += pr.alpha * I.kb[j];
    } else {
      I.lam[j - I.n_x] += pr.alpha * I.kb[j];
    }
  }
}

// ---- batched launchers -------------------------------------------------------------
cudaError_t launch_init_point_b(const DevInst* insts, const int* act, int A, double k1, double k2,
                                cudaStream_t st) {
  if (A == 0) return cudaSuccess;
  count_launch();
  k_init_point_b<<<A, 128, 0, st>>>(insts, act, k1, k2);
  return cudaGetLastError();
}

cudaError_t launch_sweep_b(const DevInst* insts, const int* act_warp, int A_warp,
                           size_t smem_warp, const int* act_cta, int A_cta, size_t smem_cta,
                           cudaStream_t st) {
  if (A_warp > 0) {
    if (smem_warp > SMEM_OPTIN_ABOVE)
      cudaFuncSetAttribute(k_sweep_warp_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_warp);
    count_launch();
    k_sweep_warp_b<<<A_warp, 32, smem_warp, st>>>(insts, act_warp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (A_cta > 0) {
    if (smem_cta > SMEM_OPTIN_ABOVE)
      cudaFuncSetAttribute(k_sweep_cta_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cta);
    count_launch();
    k_sweep_cta_b<<<A_cta, SWEEP_BS, smem_cta, st>>>(insts, act_cta);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

cudaError_t launch_theta_prep_b(const DevInst* insts, const int* act, int A, const InstParams* prm,
                                cudaStream_t st) {
  if (A == 0) return cudaSuccess;
  count_launch();
  k_theta_prep_b<<<A, IBS, 0, st>>>(insts, act, prm);
  return cudaGetLastError();
}

cudaError_t launch_vec_reduce_b(const DevInst* insts, const int* act, int A, int which,
                                cudaStream_t st) {
  if (A == 0) return cudaSuccess;
  count_launch();
  k_vec_reduce_b<<<A, IBS, 0, st>>>(insts, act, which);
  return cudaGetLastError();
}

cudaError_t launch_theta_step_b(const DevInst* insts, const int* act, int A, const InstParams* prm,
                                cudaStream_t st) {
  if (A == 0) return cudaSuccess;
  count_launch();
  k_theta_step_b<<<A, IBS, 0, st>>>(insts, act, prm);
  return cudaGetLastError();
}

cudaError_t launch_trial_barrier_b(const DevInst* insts, const int* act, int A,
                                   const InstParams* prm, cudaStream_t st) {
  if (A == 0) return cudaSuccess;
  count_launch();
  k_trial_barrier_b<<<A, IBS, 0, st>>>(insts, act, prm);
  return cudaGetLastError();
}

cudaError_t launch_update_b(const DevInst* insts, const int* act, int A, const long long* pre,
                            long long total, const InstParams* prm, int mode, cudaStream_t st) {
  if (A == 0 || total == 0) return cudaSuccess;
  int g = (int)std::min<long long>((total + 255) / 256, 8192);
  count_launch();
  k_update_b<<<std::max(g, 1), 256, 0, st>>>(insts, act, A, pre, prm, mode);
  return cudaGetLastError();
}

}  // namespace collo
