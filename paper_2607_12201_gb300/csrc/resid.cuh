// Structured FP64 KKT products and residual norms of one instance, shared by
// the evaluation kernels and the fused refinement kernel.  The reductions are
// fixed trees (sums) or maxima, so a result does not depend on which kernel or
// block size computes it.
#pragma once
#include "collo_internal.cuh"

namespace collo {

constexpr int EVAL_BS = 128;
constexpr int RED_BS = 256;

// Deterministic block reductions (fixed tree over a fixed thread order).
template <int BS>
__device__ inline double block_sum(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
#pragma unroll
  for (int s = BS / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

template <int BS>
__device__ inline double block_max(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
#pragma unroll
  for (int s = BS / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] = fmax(sh[t], sh[t + s]);
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// Structured FP64 product y = K v of the regularised KKT matrix
//   [ W + diag(sigma) + dw I   J^T  ] [vx]
//   [ J                       -dc I ] [vl]
// and r = b - y (b may be null: r = -y).  The derivative blocks are visited
// only at their structural nonzeros (the pattern lists of DevProb, ascending,
// so each sum keeps the order of the dense loop; the skipped terms are exact
// zeros).  One block per element computes the
// element's 2 (K + 1) n rows and its contribution to the p parameter rows; norms per
// element go to npart[i][0..2] (max |r_x|, max |r_c|, max |b| over the
// element's rows).
template <int BS = EVAL_BS>
__device__ inline void resid_elem(const DevProb& P, const DevEval& E, const double* __restrict__ sigma,
                           double dw, double dc, const double* __restrict__ vx,
                           const double* __restrict__ vl, const double* __restrict__ bx,
                           double bxs, const double* __restrict__ bc, double bcs,
                           double* __restrict__ rout, double* __restrict__ thpart,
                           double* __restrict__ npart, int i, double* red) {
  const int n = P.n, p = P.p, N = P.N, K = P.K, np = P.np;
  const int tid = threadIdx.x;
  const size_t nz = (size_t)N * np * n, nx = nz + p;
  const size_t zoff = (size_t)i * np * n;
  const double* vz = vx;
  const double* vt = vx ? vx + nz : nullptr;
  const size_t nn = (size_t)n * n, np_ = (size_t)n * p;
  const double* JZ = E.JZ + (size_t)i * K * nn;
  const double* JT = E.JT + (size_t)i * K * np_;
  const double* Wzz = E.Wzz + (size_t)i * K * nn;
  const double* Wzt = E.Wzt + (size_t)i * K * np_;
  const double* Wob = E.Wobj + (size_t)i * n * np * np;
  const bool next = chain_next(P, i);
  double mx = 0.0, mc = 0.0, mb = 0.0;
  for (int idx = tid; idx < np * n; idx += BS) {
    const int j = idx / n, s = idx - j * n;
    // primal row z[i][j][s]
    double y = 0.0;
    if (vz) {
      if (P.obs_sp[s])
        for (int l = 0; l < np; ++l) y += Wob[(s * np + j) * np + l] * vz[zoff + l * n + s];
      if (j >= 1) {
        const double* wr = Wzz + (size_t)(j - 1) * nn + (size_t)s * n;
        for (int e = P.wzr_ptr[s]; e < P.wzr_ptr[s + 1]; ++e) {
          const int t = P.wzr_i[e];
          y += wr[t] * vz[zoff + j * n + t];
        }
        const double* wt = Wzt + (size_t)(j - 1) * np_ + (size_t)s * p;
        for (int e = P.wtr_ptr[s]; e < P.wtr_ptr[s + 1]; ++e) {
          const int q = P.wtr_i[e];
          y += wt[q] * vt[q];
        }
      }
      y += ((sigma ? sigma[zoff + idx] : 0.0) + dw) * vz[zoff + idx];
    }
    if (vl) {
      if (j >= 1) {
        const double* jz = JZ + (size_t)(j - 1) * nn;
        for (int e = P.jzc_ptr[s]; e < P.jzc_ptr[s + 1]; ++e) {
          const int t = P.jzc_i[e];
          y += jz[(size_t)t * n + s] * vl[zoff + j * n + t];
        }
      }
      for (int k = 1; k < np; ++k) y += P.D[k][j] * vl[zoff + k * n + s];
      if (j == 0) y += vl[zoff + s];
      // the next element's continuity row: -b_j (Radau: -1 at j = K)
      if (next && P.bw[j] != 0.0) {
        if (P.gauss) y -= P.bw[j] * vl[zoff + np * n + s];
        else y -= vl[zoff + np * n + s];
      }
    }
    if (bx) mb = fmax(mb, fabs(bx[zoff + idx]));
    if (bc) mb = fmax(mb, fabs(bc[zoff + idx]));
    double rr = (bx ? bxs * bx[zoff + idx] : 0.0) - y;
    if (rout) rout[zoff + idx] = rr;
    mx = fmax(mx, fabs(rr));
    // dual row c[i][j][s]
    double yc = 0.0;
    if (vz) {
      if (j == 0) {
        double prev = 0.0;
        if (!chain_start(P, i)) {
          if (!P.gauss) {
            prev = vz[zoff - n + s];
          } else {
            const size_t po = zoff - (size_t)np * n + s;
            for (int l = 0; l < np; ++l) prev += P.bw[l] * vz[po + (size_t)l * n];
          }
        }
        yc = vz[zoff + s] - prev;
      } else {
        for (int l = 0; l < np; ++l) yc += P.D[j][l] * vz[zoff + l * n + s];
        const double* jz = JZ + (size_t)(j - 1) * nn + (size_t)s * n;
        for (int e = P.jzr_ptr[s]; e < P.jzr_ptr[s + 1]; ++e) {
          const int t = P.jzr_i[e];
          yc += jz[t] * vz[zoff + j * n + t];
        }
        const double* jt = JT + (size_t)(j - 1) * np_ + (size_t)s * p;
        for (int e = P.jtr_ptr[s]; e < P.jtr_ptr[s + 1]; ++e) {
          const int q = P.jtr_i[e];
          yc += jt[q] * vt[q];
        }
      }
    }
    if (vl) yc -= dc * vl[zoff + idx];
    double rc = (bc ? bcs * bc[zoff + idx] : 0.0) - yc;
    if (rout) rout[nx + zoff + idx] = rc;
    mc = fmax(mc, fabs(rc));
  }
  // this element's part of the parameter rows
  for (int q = tid; q < p; q += BS) {
    double y = 0.0;
    for (int k = 1; k < np; ++k)
      for (int e = P.thq_ptr[q]; e < P.thq_ptr[q + 1]; ++e) {
        const int s = P.thq_i[e];
        if (vz) y += Wzt[(size_t)(k - 1) * np_ + (size_t)s * p + q] * vz[zoff + k * n + s];
        if (vl) y += JT[(size_t)(k - 1) * np_ + (size_t)s * p + q] * vl[zoff + k * n + s];
      }
    thpart[(size_t)i * p + q] = y;
  }
  mx = block_max<BS>(mx, red);
  mc = block_max<BS>(mc, red);
  mb = block_max<BS>(mb, red);
  if (tid == 0) { npart[i * 3 + 0] = mx; npart[i * 3 + 1] = mc; npart[i * 3 + 2] = mb; }
}

// Residual modes of the batched product (which vectors of the instance):
//   R_DUAL: r_x = -(grad + J^T lambda - zl + zu)   (dual infeasibility)
//   R_RHS:  Newton right-hand side -[grad phi_mu + J^T lambda; c] into ka
//   R_IR:   r = ka - K kb with the factorization's sigma / delta_w / delta_c into kr
enum ResidMode { R_DUAL = 0, R_RHS = 1, R_IR = 2 };

struct ResidArgs {
  const double *sigma, *vx, *vl, *bx, *bc, *th_extra;
  double bxs, bcs, dw, dc;
  double* rout;
};

__device__ inline ResidArgs resid_args(const DevInst& I, const InstParams& pr, int mode) {
  ResidArgs a{};
  if (mode == R_DUAL) {
    a.vl = I.lam; a.bx = I.E.grad; a.bxs = -1.0; a.th_extra = I.zlmzu;
  } else if (mode == R_RHS) {
    a.vl = I.lam; a.bx = I.E.grad; a.bxs = -1.0; a.bc = I.E.c; a.bcs = -1.0;
    a.th_extra = I.bar; a.rout = I.ka;
  } else {
    a.sigma = I.sigma; a.vx = I.kb; a.vl = I.kb + I.n_x; a.bx = I.ka; a.bxs = 1.0;
    a.bc = I.ka + I.n_x; a.bcs = 1.0; a.dw = pr.dw; a.dc = pr.dc; a.rout = I.kr;
  }
  return a;
}

// Parameter rows of r = b - K v, and the global norms:
// out[0] = max|r_x|, out[1] = max|r_c|, out[2] = max|b| (b may be null).
// The element contributions thpart[N][p] are summed by warp w for the
// columns q = w, w + 8, ...: lane-strided partial sums, then a fixed
// shuffle tree.
__device__ inline void resid_theta_one(const DevProb& P, const DevEval& E,
                                const double* __restrict__ sigma, double dw,
                                const double* __restrict__ vx, const double* __restrict__ bx,
                                double bxs, const double* __restrict__ bc,
                                double* __restrict__ rout, const double* __restrict__ thpart,
                                const double* __restrict__ npart,
                                const double* __restrict__ th_extra, double* __restrict__ out,
                                double* sh) {
  const int tid = threadIdx.x, p = P.p, N = P.N;
  const int lane = tid & 31, warp = tid >> 5;
  const size_t nz = (size_t)N * P.np * P.n;
  double mx = 0.0, mc = 0.0, mb = 0.0;
  for (int q = warp; q < p; q += RED_BS / 32) {
    double y = 0.0;
    for (int i = lane; i < N; i += 32) y += thpart[(size_t)i * p + q];
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    if (lane == 0) {
      if (vx) y += (E.wtt[q] + (sigma ? sigma[nz + q] : 0.0) + dw) * vx[nz + q];
      if (th_extra) y -= th_extra[q];
      const double rr = (bx ? bxs * bx[nz + q] : 0.0) - y;
      if (rout) rout[nz + q] = rr;
      mx = fmax(mx, fabs(rr));
    }
  }
  for (int i = tid; i < N; i += RED_BS) {
    mx = fmax(mx, npart[i * 3 + 0]);
    mc = fmax(mc, npart[i * 3 + 1]);
    mb = fmax(mb, npart[i * 3 + 2]);
  }
  if (bx)
    for (int q = tid; q < p; q += RED_BS) mb = fmax(mb, fabs(bx[nz + q]));
  mx = block_max<RED_BS>(mx, sh);
  mc = block_max<RED_BS>(mc, sh);
  mb = block_max<RED_BS>(mb, sh);
  if (tid == 0) { out[0] = mx; out[1] = mc; out[2] = mb; }
}

}  // namespace collo
