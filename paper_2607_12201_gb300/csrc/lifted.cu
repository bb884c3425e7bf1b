// Relaxed-equality ("lifted") condensed-space Newton step: the KKT form of the
// paper's solver configuration (Section "Optimization framework
// configurations", MadNLP's LiftedKKT; Introduction: a KKT system that
// factorizes without pivoting).
//
// The equalities c(x) = 0 are relaxed to -r <= c(x) <= r with slacks
// s = c(x); with Sigma_s the slacks' barrier diagonal and d = Sigma_s + dw the
// primal-dual system in (dx, ds, dlam)
//   [ W + Sigma_x + dw I   0    J^T ] [dx  ]   [r_x]
//   [ 0                    d    -I  ] [ds  ] = [r_s]
//   [ J                   -I     0  ] [dlam]   [r_c]
// condenses to the primal system Kc dx = r_x + J^T (d r_c + r_s) with
//   Kc = W + Sigma_x + dw I + J^T diag(d) J,
// ds = J dx - r_c, dlam = d ds - r_s.  Kc is positive definite exactly when the
// full system has the inertia an interior-point step needs, so it is factored
// by Cholesky without pivoting and a non-positive pivot is the signal to
// raise dw.
//
// Structure on the collocation NLP: element i's variables are its points
// z_i0..z_iK; its collocation rows couple them with theta, and the continuity
// row of element i+1 couples them with z_(i+1)0.  Element i's block of Kc, in
// the local order [interior z_i1..z_iK (Kn) | z_i0 (n) | z_(i+1)0 (n) | theta (p)],
// holds W_i, the diagonal terms, and G_i^T diag(d) G_i over its collocation
// rows and outgoing continuity row G_i (the initial condition of a chain's
// first element adds d on z_i0), assembled entry by entry from the rows'
// structure and kept in packed lower storage.  The tree of eliminations:
//   1. each element's interior by Cholesky (one block per element, in shared
//      memory when the packed block fits, else in its global storage), leaving
//      a Schur complement on (z_i0, z_(i+1)0, theta);
//   2. the chain of n x n blocks over z_i0 (coupled to its successor) by block
//      cyclic reduction with Cholesky pivots, each level one launch of
//      eliminations and one of neighbour updates;
//   3. the p x p parameter block, assembled from every element's and every
//      chain block's contribution in a fixed order, by Cholesky.
// Everything is FP64: Sigma_s reaches mu / r^2 next to W, far beyond FP32.  The
// solve runs the same tree forward and back and is refined in FP64 against
// the unreduced system (products with W and J through the structured KKT
// residual kernel).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lifted.cuh"

namespace collo {

void lifted_free(LiftedStore* L) { delete L; }

namespace {

__host__ __device__ inline size_t zflat(const DevProb& P, int i, int j, int s) {
  return ((size_t)i * P.np + j) * P.n + s;
}

// Global index of the unknown at local position a of element i's block, with
// its kind: 0 interior / own z_i0, 1 next element's z_0, 2 theta.
__device__ inline void local_decode(const DevProb& P, int kn, int a, int& pt, int& s, int& kind) {
  const int n = P.n;
  if (a < kn) { pt = a / n + 1; s = a - (pt - 1) * n; kind = 0; }
  else if (a < kn + n) { pt = 0; s = a - kn; kind = 0; }
  else if (a < kn + 2 * n) { pt = 0; s = a - kn - n; kind = 1; }
  else { pt = -1; s = a - kn - 2 * n; kind = 2; }
}

// Packed lower-triangular storage of a symmetric block: row r holds columns
// 0..r at tri(r).
__host__ __device__ inline size_t tri(int r) { return (size_t)r * (r + 1) / 2; }

// Coefficient of own point j in the outgoing continuity row (Eq. 2c).
__device__ inline double cont_coef(const DevProb& P, int j) {
  if (P.gauss) return -P.bw[j];
  return j == P.K ? -1.0 : 0.0;
}

// Entry (a, b), a >= b, of element i's block of Kc before elimination, from
// the structure of its constraint rows: collocation row (k, t) has D[k][j] on
// point j != k of species t, the node block M_k = D[k][k] I + JZ_k on point k
// and JT_k on theta; the outgoing continuity row of species s has -b_j on the
// element's points and 1 on the next element's z_0.  So J^T diag(d) J needs,
// per entry, K terms and one length-n sum over the node block where both
// columns sit on the same point.
__device__ inline double elem_entry(const DevProb& P, const DevEval& E, const double* __restrict__ d,
                                    const double* __restrict__ sigx, double dw, int i, int kn,
                                    int a, int b) {
  const int n = P.n, np = P.np, K = P.K, p = P.p;
  int pa, sa, ka, pb, sb, kb;
  local_decode(P, kn, a, pa, sa, ka);
  local_decode(P, kn, b, pb, sb, kb);
  const double* __restrict__ JZ = E.JZ + (size_t)i * K * n * n;   // [k-1][t][s]
  const double* __restrict__ JT = E.JT + (size_t)i * K * n * p;   // [k-1][t][q]
  const double* __restrict__ dk = d + zflat(P, i, 0, 0);         // [k][t]
  auto M = [&](int k, int t, int c) {
    return JZ[((size_t)(k - 1) * n + t) * n + c] + (t == c ? P.D[k][k] : 0.0);
  };
  double v = 0.0;
  if (ka == 0 && kb == 0) {
    for (int k = 1; k <= K; ++k) {
      if (pa != k && pb != k) {
        if (sa == sb) v += P.D[k][pa] * P.D[k][pb] * dk[k * n + sa];
      } else if (pa != k) {
        v += P.D[k][pa] * dk[k * n + sa] * M(k, sa, sb);
      } else if (pb != k) {
        v += P.D[k][pb] * dk[k * n + sb] * M(k, sb, sa);
      } else {
        for (int t = 0; t < n; ++t) v += dk[k * n + t] * M(k, t, sa) * M(k, t, sb);
      }
    }
    if (sa == sb) v += E.Wobj[(((size_t)i * n + sa) * np + pa) * np + pb];
    if (pa == pb && pa >= 1) v += E.Wzz[(((size_t)i * K + (pa - 1)) * n + sa) * n + sb];
    if (a == b) {
      v += dw + sigx[zflat(P, i, pa, sa)];
      if (pa == 0 && chain_start(P, i)) v += d[zflat(P, i, 0, sa)];
    }
  } else if (ka == 2 && kb == 0) {
    for (int k = 1; k <= K; ++k) {
      if (pb != k) {
        v += P.D[k][pb] * dk[k * n + sb] * JT[((size_t)(k - 1) * n + sb) * p + sa];
      } else {
        for (int t = 0; t < n; ++t)
          v += dk[k * n + t] * JT[((size_t)(k - 1) * n + t) * p + sa] * M(k, t, sb);
      }
    }
    if (pb >= 1) v += E.Wzt[(((size_t)i * K + (pb - 1)) * n + sb) * p + sa];
  } else if (ka == 2 && kb == 2) {
    for (int k = 1; k <= K; ++k)
      for (int t = 0; t < n; ++t)
        v += dk[k * n + t] * JT[((size_t)(k - 1) * n + t) * p + sa] *
             JT[((size_t)(k - 1) * n + t) * p + sb];
  }
  if (ka != 2 && kb != 2 && sa == sb && chain_next(P, i)) {
    const double ga = ka == 1 ? 1.0 : cont_coef(P, pa);
    const double gb = kb == 1 ? 1.0 : cont_coef(P, pb);
    v += d[zflat(P, i + 1, 0, sa)] * ga * gb;
  }
  return v;
}

// Right-looking Cholesky of the leading `cols` columns of an order-m block in
// packed lower storage (shared or global memory); col: m doubles of shared
// scratch.  Every thread of the block takes part.
__device__ inline void chol_cols_packed(double* A, int m, int cols, double* col, int* flag) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5,
            nw = nt >> 5;
  for (int c = 0; c < cols; ++c) {
    if (tid == 0) {
      const double pv = A[tri(c) + c];
      if (!(pv > 0.0)) *flag = 1;
      A[tri(c) + c] = sqrt(pv);
    }
    __syncthreads();
    const double inv = 1.0 / A[tri(c) + c];
    for (int r = c + 1 + tid; r < m; r += nt) {
      const double v = A[tri(r) + c] * inv;
      A[tri(r) + c] = v;
      col[r] = v;
    }
    __syncthreads();
    for (int r = c + 1 + warp; r < m; r += nw) {
      const double lr = col[r];
      double* row = A + tri(r);
      for (int q = c + 1 + lane; q <= r; q += 32) row[q] -= lr * col[q];
    }
    __syncthreads();
  }
}

// Right-looking Cholesky of the leading `cols` columns of the lower triangle
// of an order-m row-major block A (shared or global memory); col: m doubles
// of shared scratch.  Every thread of the block takes part.
__device__ inline void chol_cols(double* A, int m, int cols, double* col, int* flag) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5,
            nw = nt >> 5;
  for (int c = 0; c < cols; ++c) {
    if (tid == 0) {
      const double pv = A[(size_t)c * m + c];
      if (!(pv > 0.0)) *flag = 1;
      A[(size_t)c * m + c] = sqrt(pv);
    }
    __syncthreads();
    const double inv = 1.0 / A[(size_t)c * m + c];
    for (int r = c + 1 + tid; r < m; r += nt) {
      const double v = A[(size_t)r * m + c] * inv;
      A[(size_t)r * m + c] = v;
      col[r] = v;
    }
    __syncthreads();
    for (int r = c + 1 + warp; r < m; r += nw) {
      const double lr = col[r];
      double* row = A + (size_t)r * m;
      for (int q = c + 1 + lane; q <= r; q += 32) row[q] -= lr * col[q];
    }
    __syncthreads();
  }
}

// ---- factorization ----------------------------------------------------------------

// Assemble element i's block of Kc (packed lower) and eliminate its interior.
// EBS threads: 512 for blocks above 128 unknowns (one block per SM; the
// Cholesky's column steps are barrier-bound and more warps keep the FP64 pipe
// busier), 256 below (two blocks per SM).
template <int EBS>
__global__ void __launch_bounds__(EBS) k_lifted_elem(DevProb P, DevEval E, DevLifted L) {
  extern __shared__ double sm[];
  const int me = L.me, kn = L.kn, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t msz = tri(me);
  for (int i = blockIdx.x; i < P.N; i += gridDim.x) {
    double* A = L.elem_smem ? sm : L.blk + (size_t)i * msz;
    double* col = L.elem_smem ? sm + msz : sm;
    for (int a = warp; a < me; a += EBS / 32)
      for (int b = lane; b <= a; b += 32)
        A[tri(a) + b] = elem_entry(P, E, L.d, L.sigx, L.dw, i, kn, a, b);
    __syncthreads();
    chol_cols_packed(A, me, kn, col, L.flag);
    if (L.elem_smem) {
      double* dst = L.blk + (size_t)i * msz;
      for (size_t idx = tid; idx < msz; idx += EBS) dst[idx] = A[idx];
    }
    __syncthreads();
  }
}

__device__ inline double lower_at(const double* A, int r, int c) {
  return r >= c ? A[tri(r) + c] : A[tri(c) + r];
}

// Chain blocks from the elements' frontal Schur complements.
__global__ void __launch_bounds__(LBS) k_lifted_chain(DevProb P, DevLifted L) {
  const int i = blockIdx.x, n = P.n, p = P.p, me = L.me, kn = L.kn;
  const size_t msz = tri(me);
  const double* Bi = L.blk + (size_t)i * msz;
  const bool prev = i > 0 && chain_next(P, i - 1);
  const double* Bp = prev ? L.blk + (size_t)(i - 1) * msz : nullptr;
  const bool next = chain_next(P, i);
  for (int idx = threadIdx.x; idx < n * n; idx += LBS) {
    const int s = idx / n, t = idx - s * n;
    double v = lower_at(Bi, kn + s, kn + t);
    if (prev) v += lower_at(Bp, kn + n + s, kn + n + t);
    L.Dg[(size_t)i * n * n + idx] = v;
    L.Cp[(size_t)i * n * n + idx] = next ? Bi[tri(kn + n + s) + kn + t] : 0.0;
  }
  for (int idx = threadIdx.x; idx < n * p; idx += LBS) {
    const int s = idx / p, q = idx - s * p;
    double v = Bi[tri(kn + 2 * n + q) + kn + s];
    if (prev) v += Bp[tri(kn + 2 * n + q) + kn + n + s];
    L.Bd[(size_t)i * n * p + idx] = v;
  }
}

// Eliminated chain block of a reduction level: blockIdx.x-th j with
// j = 2^lv (2 blockIdx.x + 1), or j = 0 when `last`.
__device__ inline int elim_index(int lv, int b, bool last) {
  return last ? 0 : (2 * b + 1) << lv;
}

// Cholesky of chain block j and X = L_j^-1 [M_ja | M_jb | B_j].
__global__ void __launch_bounds__(LBS) k_lifted_bcr_elim(DevProb P, DevLifted L, int lv,
                                                          int last) {
  extern __shared__ double sm[];
  const int n = P.n, p = P.p, N = P.N, tid = threadIdx.x, cw = L.cw;
  const int j = elim_index(lv, blockIdx.x, last);
  const int h = 1 << lv;
  const bool has_a = !last, has_b = !last && j + h < N;
  double* Ls = sm;                       // n x n
  double* buf = sm + (size_t)n * n;      // n x cw
  double* col = buf + (size_t)n * cw;    // n
  const double* Dj = L.Dg + (size_t)j * n * n;
  for (int idx = tid; idx < n * n; idx += LBS) Ls[idx] = Dj[idx];
  __syncthreads();
  chol_cols(Ls, n, n, col, L.flag);
  for (int idx = tid; idx < n * n; idx += LBS) L.Dg[(size_t)j * n * n + idx] = Ls[idx];
  // right-hand-side columns: [0, n) coupling to a, [n, 2n) to b, [2n, 2n + p) border
  const int ncol = 2 * n + p;
  const double* Ca = has_a ? L.Cp + (size_t)(j - h) * n * n : nullptr;   // rows j, cols a
  const double* Cb = has_b ? L.Cp + (size_t)j * n * n : nullptr;         // rows b, cols j
  const double* Bj = L.Bd + (size_t)j * n * p;
  for (int c0 = 0; c0 < ncol; c0 += cw) {
    const int c = c0 + tid;
    const bool own = tid < cw && c < ncol;
    if (own) {
      for (int r = 0; r < n; ++r) {
        double m;
        if (c < n) m = has_a ? Ca[(size_t)r * n + c] : 0.0;
        else if (c < 2 * n) m = has_b ? Cb[(size_t)(c - n) * n + r] : 0.0;
        else m = Bj[(size_t)r * p + (c - 2 * n)];
        for (int k = 0; k < r; ++k) m -= Ls[r * n + k] * buf[k * cw + tid];
        buf[r * cw + tid] = m / Ls[r * n + r];
      }
      for (int r = 0; r < n; ++r) {
        const double v = buf[r * cw + tid];
        if (c < n) L.Xa[((size_t)j * n + r) * n + c] = v;
        else if (c < 2 * n) L.Xb[((size_t)j * n + r) * n + (c - n)] = v;
        else L.Xt[((size_t)j * n + r) * p + (c - 2 * n)] = v;
      }
    }
  }
}

// Surviving chain block a = 2^(lv+1) blockIdx.x after the eliminations of lv.
__global__ void __launch_bounds__(LBS) k_lifted_bcr_update(DevProb P, DevLifted L, int lv) {
  const int n = P.n, p = P.p, N = P.N, h = 1 << lv;
  const int a = blockIdx.x << (lv + 1);
  const int jl = a - h, jr = a + h;
  const bool hl = a > 0, hr = jr < N, hb = hr && jr + h < N;
  const double* Xbl = hl ? L.Xb + (size_t)jl * n * n : nullptr;
  const double* Xtl = hl ? L.Xt + (size_t)jl * n * p : nullptr;
  const double* Xar = hr ? L.Xa + (size_t)jr * n * n : nullptr;
  const double* Xbr = hr ? L.Xb + (size_t)jr * n * n : nullptr;
  const double* Xtr = hr ? L.Xt + (size_t)jr * n * p : nullptr;
  for (int idx = threadIdx.x; idx < n * n; idx += LBS) {
    const int s = idx / n, t = idx - s * n;
    double v = 0.0, w = 0.0;
    for (int k = 0; k < n; ++k) {
      if (hl) v += Xbl[k * n + s] * Xbl[k * n + t];
      if (hr) v += Xar[k * n + s] * Xar[k * n + t];
      if (hb) w += Xbr[k * n + s] * Xar[k * n + t];
    }
    L.Dg[(size_t)a * n * n + idx] -= v;
    L.Cp[(size_t)a * n * n + idx] = hb ? -w : 0.0;
  }
  for (int idx = threadIdx.x; idx < n * p; idx += LBS) {
    const int s = idx / p, q = idx - s * p;
    double v = 0.0;
    for (int k = 0; k < n; ++k) {
      if (hl) v += Xbl[k * n + s] * Xtl[k * p + q];
      if (hr) v += Xar[k * n + s] * Xtr[k * p + q];
    }
    L.Bd[(size_t)a * n * p + idx] -= v;
  }
}

// Partial sums of the parameter block over a chunk of elements / chain
// blocks: each element's frontal theta-theta entry minus the chain block's
// X_theta^T X_theta.
__global__ void __launch_bounds__(LBS) k_lifted_theta_part(DevProb P, DevLifted L) {
  const int p = P.p, n = P.n, N = P.N, me = L.me, kn = L.kn;
  const int idx = blockIdx.x * LBS + threadIdx.x;
  if (idx >= p * p) return;
  const int q1 = idx / p, q2 = idx - q1 * p;
  if (q2 > q1) return;
  const int c = blockIdx.y, per = (N + L.chunks - 1) / L.chunks;
  const int i0 = c * per, i1 = min(N, i0 + per);
  double v = 0.0;
  for (int i = i0; i < i1; ++i) {
    v += L.blk[(size_t)i * tri(me) + tri(kn + 2 * n + q1) + kn + 2 * n + q2];
    const double* X = L.Xt + (size_t)i * n * p;
    double t = 0.0;
    for (int s = 0; s < n; ++s) t += X[s * p + q1] * X[s * p + q2];
    v -= t;
  }
  L.Spart[(size_t)c * p * p + idx] = v;
}

__global__ void __launch_bounds__(LBS) k_lifted_theta_sum(DevProb P, DevEval E, DevLifted L) {
  const int p = P.p;
  const int idx = blockIdx.x * LBS + threadIdx.x;
  if (idx >= p * p) return;
  const int q1 = idx / p, q2 = idx - q1 * p;
  if (q2 > q1) return;
  double v = 0.0;
  for (int c = 0; c < L.chunks; ++c) v += L.Spart[(size_t)c * p * p + idx];
  if (q1 == q2) {
    const size_t nz = (size_t)P.N * P.np * P.n;
    v += E.wtt[q1] + L.sigx[nz + q1] + L.dw;
  }
  L.S[idx] = v;
}

__global__ void __launch_bounds__(1024) k_lifted_theta_chol(DevProb P, DevLifted L, int in_smem) {
  extern __shared__ double sm[];
  const int p = P.p;
  double* A = in_smem ? sm : L.S;
  double* col = in_smem ? sm + (size_t)p * p : L.Spart;   // p doubles of scratch
  if (in_smem) {
    for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) A[idx] = L.S[idx];
    __syncthreads();
  }
  chol_cols(A, p, p, col, L.flag);
  if (in_smem)
    for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) L.S[idx] = A[idx];
}

// ---- solve ------------------------------------------------------------------------

__global__ void __launch_bounds__(LBS) k_lifted_rhs(DevLifted L, const double* __restrict__ rs,
                                                     const double* __restrict__ rc, size_t nc) {
  for (size_t r = blockIdx.x * (size_t)LBS + threadIdx.x; r < nc; r += (size_t)gridDim.x * LBS)
    L.vneg[r] = -(L.d[r] * rc[r] + rs[r]);
}

// Forward substitution through element i's interior: y_I = L_II^-1 b_I and the
// element's contributions -L_FI y_I to the frontal right-hand side.
__global__ void __launch_bounds__(LBS) k_lifted_fwd_elem(DevProb P, DevLifted L,
                                                          const double* __restrict__ b) {
  extern __shared__ double sm[];
  const int me = L.me, kn = L.kn, n = P.n, tid = threadIdx.x;
  double* y = sm;
  for (int i = blockIdx.x; i < P.N; i += gridDim.x) {
    const double* A = L.blk + (size_t)i * tri(me);
    for (int a = tid; a < me; a += LBS)
      y[a] = a < kn ? b[zflat(P, i, a / n + 1, a % n)] : 0.0;
    __syncthreads();
    for (int c = 0; c < kn; ++c) {
      const double yc = y[c] / A[tri(c) + c];
      __syncthreads();
      if (tid == 0) y[c] = yc;
      for (int r = c + 1 + tid; r < me; r += LBS) y[r] -= A[tri(r) + c] * yc;
      __syncthreads();
    }
    for (int a = tid; a < me; a += LBS) {
      if (a < kn) L.y[zflat(P, i, a / n + 1, a % n)] = y[a];
      else L.ue[(size_t)i * (me - kn) + (a - kn)] = y[a];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(LBS) k_lifted_chain_rhs(DevProb P, DevLifted L,
                                                           const double* __restrict__ b) {
  const int n = P.n, F = L.me - L.kn;
  const size_t tot = (size_t)P.N * n;
  for (size_t idx = blockIdx.x * (size_t)LBS + threadIdx.x; idx < tot;
       idx += (size_t)gridDim.x * LBS) {
    const int i = (int)(idx / n), s = (int)(idx - (size_t)i * n);
    double v = b[zflat(P, i, 0, s)] + L.ue[(size_t)i * F + s];
    if (i > 0 && chain_next(P, i - 1)) v += L.ue[(size_t)(i - 1) * F + n + s];
    L.cc[idx] = v;
  }
}

// Forward substitution with chain block j's factor: w_j = L_j^-1 c_j (one warp).
__global__ void __launch_bounds__(32) k_lifted_bcr_fwd(DevProb P, DevLifted L, int lv, int last) {
  const int n = P.n, lane = threadIdx.x;
  const int j = elim_index(lv, blockIdx.x, last);
  const double* Lj = L.Dg + (size_t)j * n * n;
  double* c = L.cc + (size_t)j * n;
  for (int r = 0; r < n; ++r) {
    double part = 0.0;
    for (int k = lane; k < r; k += 32) part += Lj[r * n + k] * c[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    __syncwarp();
    if (lane == 0) c[r] = (c[r] - part) / Lj[r * n + r];
    __syncwarp();
  }
}

__global__ void __launch_bounds__(LBS) k_lifted_bcr_fwd_update(DevProb P, DevLifted L, int lv) {
  const int n = P.n, N = P.N, h = 1 << lv;
  const int a = blockIdx.x << (lv + 1);
  const int jl = a - h, jr = a + h;
  const bool hl = a > 0, hr = jr < N;
  for (int s = threadIdx.x; s < n; s += LBS) {
    double v = 0.0;
    for (int k = 0; k < n; ++k) {
      if (hl) v += L.Xb[((size_t)jl * n + k) * n + s] * L.cc[(size_t)jl * n + k];
      if (hr) v += L.Xa[((size_t)jr * n + k) * n + s] * L.cc[(size_t)jr * n + k];
    }
    L.cc[(size_t)a * n + s] -= v;
  }
}

// Partial sums of the parameter right-hand side over a chunk of elements /
// chain blocks: sum_i (ue_i,theta - Xt_i^T w_i).
__global__ void __launch_bounds__(LBS) k_lifted_theta_rhs_part(DevProb P, DevLifted L) {
  const int p = P.p, n = P.n, N = P.N, F = L.me - L.kn;
  const int c = blockIdx.x, per = (N + L.chunks - 1) / L.chunks;
  const int i0 = c * per, i1 = min(N, i0 + per);
  for (int q = threadIdx.x; q < p; q += LBS) {
    double v = 0.0;
    for (int i = i0; i < i1; ++i) {
      v += L.ue[(size_t)i * F + 2 * n + q];
      const double* X = L.Xt + (size_t)i * n * p;
      const double* w = L.cc + (size_t)i * n;
      double t = 0.0;
      for (int s = 0; s < n; ++s) t += X[s * p + q] * w[s];
      v -= t;
    }
    L.Spart[(size_t)c * p + q] = v;
  }
}

// Parameter right-hand side ct = b_theta + the chunk sums in order, then
// S xt = ct by the Cholesky factor (one block).
__global__ void __launch_bounds__(1024) k_lifted_theta_solve(DevProb P, DevLifted L,
                                                              const double* __restrict__ b) {
  extern __shared__ double sm[];
  const int p = P.p, n = P.n, N = P.N, tid = threadIdx.x;
  const size_t nz = (size_t)N * P.np * n;
  double* x = sm;
  for (int q = tid; q < p; q += blockDim.x) {
    double v = b[nz + q];
    for (int c = 0; c < L.chunks; ++c) v += L.Spart[(size_t)c * p + q];
    x[q] = v;
  }
  __syncthreads();
  const double* S = L.S;
  for (int c = 0; c < p; ++c) {          // forward: L y = ct
    const double yc = x[c] / S[(size_t)c * p + c];
    __syncthreads();
    if (tid == 0) x[c] = yc;
    for (int r = c + 1 + tid; r < p; r += blockDim.x) x[r] -= S[(size_t)r * p + c] * yc;
    __syncthreads();
  }
  for (int c = p - 1; c >= 0; --c) {     // backward: L^T x = y
    const double xc = x[c] / S[(size_t)c * p + c];
    __syncthreads();
    if (tid == 0) x[c] = xc;
    for (int r = tid; r < c; r += blockDim.x) x[r] -= S[(size_t)c * p + r] * xc;
    __syncthreads();
  }
  for (int q = tid; q < p; q += blockDim.x) L.ct[q] = x[q];
}

// Back substitution of chain block j: x_j = L_j^-T (w_j - Xa x_a - Xb x_b - Xt x_theta).
__global__ void __launch_bounds__(32) k_lifted_bcr_back(DevProb P, DevLifted L, int lv, int last) {
  extern __shared__ double sm[];
  const int n = P.n, p = P.p, N = P.N, lane = threadIdx.x, h = 1 << lv;
  const int j = elim_index(lv, blockIdx.x, last);
  const bool ha = !last, hb = !last && j + h < N;
  const double* Lj = L.Dg + (size_t)j * n * n;
  double* t = sm;
  for (int r = lane; r < n; r += 32) {
    double v = L.cc[(size_t)j * n + r];
    const double* xa = ha ? L.cc + (size_t)(j - h) * n : nullptr;
    const double* xb = hb ? L.cc + (size_t)(j + h) * n : nullptr;
    for (int k = 0; k < n; ++k) {
      if (ha) v -= L.Xa[((size_t)j * n + r) * n + k] * xa[k];
      if (hb) v -= L.Xb[((size_t)j * n + r) * n + k] * xb[k];
    }
    for (int q = 0; q < p; ++q) v -= L.Xt[((size_t)j * n + r) * p + q] * L.ct[q];
    t[r] = v;
  }
  __syncwarp();
  for (int c = n - 1; c >= 0; --c) {
    const double xc = t[c] / Lj[c * n + c];
    __syncwarp();
    for (int r = lane; r < c; r += 32) t[r] -= Lj[c * n + r] * xc;
    if (lane == 0) t[c] = xc;
    __syncwarp();
  }
  for (int r = lane; r < n; r += 32) L.cc[(size_t)j * n + r] = t[r];
}

// Back substitution through element i's interior and assembly of dx.
__global__ void __launch_bounds__(LBS) k_lifted_back_elem(DevProb P, DevLifted L,
                                                           double* __restrict__ dx) {
  extern __shared__ double sm[];
  const int me = L.me, kn = L.kn, n = P.n, p = P.p, tid = threadIdx.x;
  double* xf = sm;            // frontal solution (2n + p)
  double* t = sm + (me - kn); // interior (kn)
  for (int i = blockIdx.x; i < P.N; i += gridDim.x) {
    const double* A = L.blk + (size_t)i * tri(me);
    const bool next = chain_next(P, i);
    for (int f = tid; f < me - kn; f += LBS) {
      double v;
      if (f < n) v = L.cc[(size_t)i * n + f];
      else if (f < 2 * n) v = next ? L.cc[(size_t)(i + 1) * n + (f - n)] : 0.0;
      else v = L.ct[f - 2 * n];
      xf[f] = v;
    }
    __syncthreads();
    for (int c = tid; c < kn; c += LBS) {
      double v = L.y[zflat(P, i, c / n + 1, c % n)];
      for (int f = 0; f < me - kn; ++f) v -= A[tri(kn + f) + c] * xf[f];
      t[c] = v;
    }
    __syncthreads();
    for (int c = kn - 1; c >= 0; --c) {
      const double xc = t[c] / A[tri(c) + c];
      __syncthreads();
      if (tid == 0) t[c] = xc;
      for (int r = tid; r < c; r += LBS) t[r] -= A[tri(c) + r] * xc;
      __syncthreads();
    }
    for (int c = tid; c < kn; c += LBS) dx[zflat(P, i, c / n + 1, c % n)] = t[c];
    for (int s = tid; s < n; s += LBS) dx[zflat(P, i, 0, s)] = xf[s];
    if (i == 0)
      for (int q = tid; q < p; q += LBS) dx[(size_t)P.N * P.np * n + q] = xf[2 * n + q];
    __syncthreads();
  }
}

// ds = J dx - r_c (from res_c = r_c - J dx), dlam = d ds - r_s.
__global__ void __launch_bounds__(LBS) k_lifted_finish(DevLifted L, const double* __restrict__ resc,
                                                        const double* __restrict__ rs,
                                                        double* __restrict__ ds,
                                                        double* __restrict__ dl, size_t nc) {
  for (size_t r = blockIdx.x * (size_t)LBS + threadIdx.x; r < nc; r += (size_t)gridDim.x * LBS) {
    const double v = -resc[r];
    ds[r] = v;
    dl[r] = L.d[r] * v - rs[r];
  }
}

// Residual of the unreduced system from the structured one (res_x = r_x -
// H dx - J^T dlam, res_c = r_c - J dx): q_x = res_x, q_s = r_s - d ds + dlam,
// q_c = res_c + ds, and the norms max|q|, max|b| (one block).
__global__ void __launch_bounds__(1024) k_lifted_resid(DevLifted L, size_t nx, size_t nc) {
  __shared__ double sh[2][32];
  const int tid = threadIdx.x;
  double mq = 0.0, mb = 0.0;
  for (size_t r = tid; r < nx; r += blockDim.x) {
    const double v = L.res[r];
    L.qx[r] = v;
    mq = fmax(mq, fabs(v));
    mb = fmax(mb, fabs(L.rx[r]));
  }
  for (size_t r = tid; r < nc; r += blockDim.x) {
    const double qc = L.res[nx + r] + L.ds[r];
    const double qs = L.rs[r] - (L.d[r] * L.ds[r] - L.dl[r]);
    L.qc[r] = qc;
    L.qs[r] = qs;
    mq = fmax(mq, fmax(fabs(qc), fabs(qs)));
    mb = fmax(mb, fmax(fabs(L.rs[r]), fabs(L.rc[r])));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mq = fmax(mq, __shfl_xor_sync(0xffffffffu, mq, o));
    mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  }
  if ((tid & 31) == 0) { sh[0][tid >> 5] = mq; sh[1][tid >> 5] = mb; }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a = fmax(a, sh[0][w]); b = fmax(b, sh[1][w]); }
    L.nrm[0] = a;
    L.nrm[1] = b;
  }
}

__global__ void __launch_bounds__(LBS) k_lifted_shift(double* __restrict__ y, double a, size_t n) {
  for (size_t r = blockIdx.x * (size_t)LBS + threadIdx.x; r < n; r += (size_t)gridDim.x * LBS)
    y[r] += a;
}

__global__ void __launch_bounds__(LBS) k_lifted_add(double* __restrict__ y,
                                                     const double* __restrict__ x, size_t n) {
  for (size_t r = blockIdx.x * (size_t)LBS + threadIdx.x; r < n; r += (size_t)gridDim.x * LBS)
    y[r] += x[r];
}

int grid_of(size_t n) { return (int)std::min<size_t>((n + LBS - 1) / LBS, 4 * 152); }

// Shared memory of the element kernel: the packed block and a column.
size_t elem_smem_bytes(int me) { return (tri(me) + me) * sizeof(double); }

size_t bcr_smem_bytes(int n, int cw) { return ((size_t)n * n + (size_t)n * cw + n) * sizeof(double); }

cudaError_t set_smem(const void* f, size_t bytes) {
  if (bytes <= SMEM_OPTIN_ABOVE) return cudaSuccess;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// Storage of the lifted factorization (allocated on the first call).
collo_status lifted_storage(collo_problem* pr) {
  if (pr->lifted) return COLLO_OK;
  const DevProb& P = pr->P;
  if (bcr_smem_bytes(P.n, 32) > FACTOR_SMEM_LIMIT) {
    set_error("too many species for the lifted factorization's chain blocks");
    return COLLO_ERR_INVALID_ARG;
  }
  auto* LS = new LiftedStore();
  DevLifted* L = &LS->V;
  L->kn = P.K * P.n;
  L->me = L->kn + 2 * P.n + P.p;
  L->elem_smem = elem_smem_bytes(L->me) <= FACTOR_SMEM_LIMIT;
  L->grid_e = P.N;
  L->cw = LBS;
  while (L->cw > 32 && bcr_smem_bytes(P.n, L->cw) > FACTOR_SMEM_LIMIT) L->cw >>= 1;
  L->chunks = std::max(1, std::min(64, P.N));
  const size_t N = P.N, n = P.n, p = P.p, nx = pr->n_x, nc = pr->n_c, me = L->me;
  DevArena& m = LS->mem;
  L->sigx = m.alloc<double>(nx);
  L->d = m.alloc<double>(nc);
  L->blk = m.alloc<double>(N * tri((int)me));
  L->Dg = m.alloc<double>(N * n * n);
  L->Cp = m.alloc<double>(N * n * n);
  L->Xa = m.alloc<double>(N * n * n);
  L->Xb = m.alloc<double>(N * n * n);
  L->Bd = m.alloc<double>(N * n * p);
  L->Xt = m.alloc<double>(N * n * p);
  L->S = m.alloc<double>(p * p);
  L->Spart = m.alloc<double>((size_t)L->chunks * p * p + p);
  L->flag = m.alloc<int>(1);
  L->rx = m.alloc<double>(nx); L->rs = m.alloc<double>(nc); L->rc = m.alloc<double>(nc);
  L->dx = m.alloc<double>(nx); L->ds = m.alloc<double>(nc); L->dl = m.alloc<double>(nc);
  L->ex = m.alloc<double>(nx); L->es = m.alloc<double>(nc); L->el = m.alloc<double>(nc);
  L->qx = m.alloc<double>(nx); L->qs = m.alloc<double>(nc); L->qc = m.alloc<double>(nc);
  L->y = m.alloc<double>(nx);
  L->ue = m.alloc<double>(N * (me - L->kn));
  L->cc = m.alloc<double>(N * n);
  L->ct = m.alloc<double>(p);
  L->vneg = m.alloc<double>(nc);
  L->res = m.alloc<double>(nx + nc);
  L->nrm = m.alloc<double>(8);
  bool ok = L->sigx && L->d && L->blk && L->Dg && L->Cp && L->Xa && L->Xb && L->Bd && L->Xt &&
            L->S && L->Spart && L->flag && L->rx && L->rs && L->rc && L->dx && L->ds && L->dl &&
            L->ex && L->es && L->el && L->qx && L->qs && L->qc && L->y && L->ue && L->cc &&
            L->ct && L->vneg && L->res && L->nrm;
  if (!ok) {
    delete LS;
    set_error("out of device memory for the lifted factorization");
    return COLLO_ERR_OOM;
  }
  pr->lifted = LS;
  return COLLO_OK;
}

}  // namespace collo

using namespace collo;

namespace {

// One solve of the unreduced system through the condensed factor:
// (rx, rs, rc) -> (dx, ds, dl), all device vectors of the store.
cudaError_t lifted_solve_once(collo_problem* pr, const double* rx, const double* rs,
                              const double* rc, double* dx, double* ds, double* dl) {
  DevLifted& L = pr->lifted->V;
  const DevProb& P = pr->P;
  cudaStream_t st = pr->stream;
  const size_t nx = pr->n_x, nc = pr->n_c;
  const int n = P.n, p = P.p, N = P.N;
  cudaError_t e;
  count_launch();
  k_lifted_rhs<<<grid_of(nc), LBS, 0, st>>>(L, rs, rc, nc);
  if ((e = launch_kkt_resid(P, pr->E, L.sigx, L.dw, 0.0, nullptr, L.vneg, rx, 1.0, nullptr, 0.0,
                            L.res, pr->thpart, pr->npart, nullptr, pr->scal + 8, st)) != cudaSuccess)
    return e;
  const size_t sm_v = (size_t)L.me * sizeof(double);
  count_launch();
  k_lifted_fwd_elem<<<N, LBS, sm_v, st>>>(P, L, L.res);
  count_launch();
  k_lifted_chain_rhs<<<grid_of((size_t)N * n), LBS, 0, st>>>(P, L, L.res);
  int lv = 0;
  for (; (1 << lv) < N; ++lv) {
    const int h = 1 << lv, cnt = (N - h + 2 * h - 1) / (2 * h), surv = (N + 2 * h - 1) / (2 * h);
    count_launch(2);
    k_lifted_bcr_fwd<<<cnt, 32, 0, st>>>(P, L, lv, 0);
    k_lifted_bcr_fwd_update<<<surv, LBS, 0, st>>>(P, L, lv);
  }
  count_launch(2);
  k_lifted_bcr_fwd<<<1, 32, 0, st>>>(P, L, 0, 1);
  if (p > 0) {
    count_launch();
    k_lifted_theta_rhs_part<<<L.chunks, LBS, 0, st>>>(P, L);
  }
  k_lifted_theta_solve<<<1, 1024, (size_t)std::max(p, 1) * sizeof(double), st>>>(P, L, L.res);
  const size_t sm_n = (size_t)n * sizeof(double);
  count_launch();
  k_lifted_bcr_back<<<1, 32, sm_n, st>>>(P, L, 0, 1);
  for (int l = lv - 1; l >= 0; --l) {
    const int h = 1 << l, cnt = (N - h + 2 * h - 1) / (2 * h);
    count_launch();
    k_lifted_bcr_back<<<cnt, 32, sm_n, st>>>(P, L, l, 0);
  }
  count_launch();
  k_lifted_back_elem<<<N, LBS, sm_v, st>>>(P, L, dx);
  if ((e = launch_kkt_resid(P, pr->E, L.sigx, L.dw, 0.0, dx, nullptr, nullptr, 0.0, rc, 1.0,
                            L.res, pr->thpart, pr->npart, nullptr, pr->scal + 8, st)) != cudaSuccess)
    return e;
  count_launch();
  k_lifted_finish<<<grid_of(nc), LBS, 0, st>>>(L, L.res + nx, rs, ds, dl, nc);
  return cudaGetLastError();
}

// The factorization's kernels (element blocks, chain reduction, parameter
// block) on the store's current d and sigma_x; `elem_only`: the element
// kernel alone.  Re-running them on the same inputs reproduces the factors.
cudaError_t lifted_factor_kernels(collo_problem* pr, bool elem_only) {
  DevLifted& L = pr->lifted->V;
  const DevProb& P = pr->P;
  cudaStream_t st = pr->stream;
  const int n = P.n, p = P.p, N = P.N;
  cudaError_t e;
  const size_t sm_e = L.elem_smem ? elem_smem_bytes(L.me) : (size_t)L.me * sizeof(double);
  count_launch();
  if (L.me > 128) {
    if ((e = set_smem((const void*)k_lifted_elem<512>, sm_e)) != cudaSuccess) return e;
    k_lifted_elem<512><<<L.grid_e, 512, sm_e, st>>>(P, pr->E, L);
  } else {
    if ((e = set_smem((const void*)k_lifted_elem<256>, sm_e)) != cudaSuccess) return e;
    k_lifted_elem<256><<<L.grid_e, 256, sm_e, st>>>(P, pr->E, L);
  }
  if ((e = cudaGetLastError()) != cudaSuccess || elem_only) return e;
  count_launch();
  k_lifted_chain<<<N, LBS, 0, st>>>(P, L);
  const size_t sm_b = bcr_smem_bytes(n, L.cw);
  if ((e = set_smem((const void*)k_lifted_bcr_elim, sm_b)) != cudaSuccess) return e;
  for (int lv = 0; (1 << lv) < N; ++lv) {
    const int h = 1 << lv, cnt = (N - h + 2 * h - 1) / (2 * h), surv = (N + 2 * h - 1) / (2 * h);
    count_launch(2);
    k_lifted_bcr_elim<<<cnt, LBS, sm_b, st>>>(P, L, lv, 0);
    k_lifted_bcr_update<<<surv, LBS, 0, st>>>(P, L, lv);
  }
  count_launch();
  k_lifted_bcr_elim<<<1, LBS, sm_b, st>>>(P, L, 0, 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (p > 0) {
    const int tiles = (p * p + LBS - 1) / LBS;
    count_launch(2);
    k_lifted_theta_part<<<dim3(tiles, L.chunks), LBS, 0, st>>>(P, L);
    k_lifted_theta_sum<<<tiles, LBS, 0, st>>>(P, pr->E, L);
    const size_t sm_t = ((size_t)p * p + p) * sizeof(double);
    const int in_smem = sm_t <= FACTOR_SMEM_LIMIT;
    if ((e = set_smem((const void*)k_lifted_theta_chol, in_smem ? sm_t : 0)) != cudaSuccess)
      return e;
    count_launch();
    k_lifted_theta_chol<<<1, 1024, in_smem ? sm_t : 0, st>>>(P, L, in_smem);
  }
  return cudaGetLastError();
}

}  // namespace

namespace collo {

// Phases of the lifted path for the measurement hook: 0 the element kernel,
// 1 every factorization kernel, 2 one solve without refinement on the last
// right-hand side.  Needs a current positive-definite lifted factorization.
collo_status lifted_time_launch(collo_problem* pr, int which) {
  if (!pr->lifted || !pr->lifted->pd || pr->lifted->eval_count != pr->eval_count) {
    set_error("no positive definite lifted factorization of the current evaluation");
    return COLLO_ERR_NOT_FACTORED;
  }
  DevLifted& L = pr->lifted->V;
  if (which == 2) COLLO_CUDA(lifted_solve_once(pr, L.rx, L.rs, L.rc, L.ex, L.es, L.el));
  else COLLO_CUDA(lifted_factor_kernels(pr, which == 0));
  return COLLO_OK;
}

int lifted_grid(size_t n) { return grid_of(n); }

collo_status lifted_factor_dev(collo_problem* prob, const double* sigma_s, double dw, bool* pd) {
  LiftedStore& LS = *prob->lifted;
  DevLifted& L = LS.V;
  cudaStream_t st = prob->stream;
  const size_t nc = prob->n_c;
  L.dw = dw;
  LS.pd = false;
  LS.eval_count = -1;
  if (sigma_s != L.d)
    COLLO_CUDA(cudaMemcpyAsync(L.d, sigma_s, nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
  COLLO_CUDA(cudaMemsetAsync(L.flag, 0, sizeof(int), st));
  count_launch();
  k_lifted_shift<<<grid_of(nc), LBS, 0, st>>>(L.d, dw, nc);
  COLLO_CUDA(lifted_factor_kernels(prob, false));
  int flag = 1;
  COLLO_CUDA(cudaMemcpyAsync(&prob->hscal[48], L.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  std::memcpy(&flag, &prob->hscal[48], sizeof(int));
  LS.pd = flag == 0;
  LS.eval_count = prob->eval_count;
  *pd = LS.pd;
  return COLLO_OK;
}

collo_status lifted_solve_dev(collo_problem* prob, int refine_max, double refine_tol, int* sweeps,
                              double* relp) {
  DevLifted& L = prob->lifted->V;
  cudaStream_t st = prob->stream;
  const size_t nx = prob->n_x, nc = prob->n_c;
  COLLO_CUDA(lifted_solve_once(prob, L.rx, L.rs, L.rc, L.dx, L.ds, L.dl));
  int k = 0;
  double rel = 0.0;
  if (refine_max < 0) refine_max = 0;
  for (;;) {
    COLLO_CUDA(launch_kkt_resid(prob->P, prob->E, L.sigx, L.dw, 0.0, L.dx, L.dl, L.rx, 1.0, L.rc,
                                1.0, L.res, prob->thpart, prob->npart, nullptr, prob->scal + 8, st));
    count_launch();
    k_lifted_resid<<<1, 1024, 0, st>>>(L, nx, nc);
    COLLO_CUDA(cudaGetLastError());
    COLLO_CUDA(cudaMemcpyAsync(&prob->hscal[50], L.nrm, 2 * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
    COLLO_CUDA(cudaStreamSynchronize(st));
    rel = prob->hscal[50] / std::max(1.0, prob->hscal[51]);
    if (!(rel > refine_tol) || k >= refine_max || !std::isfinite(rel)) break;
    COLLO_CUDA(lifted_solve_once(prob, L.qx, L.qs, L.qc, L.ex, L.es, L.el));
    count_launch(3);
    k_lifted_add<<<grid_of(nx), LBS, 0, st>>>(L.dx, L.ex, nx);
    k_lifted_add<<<grid_of(nc), LBS, 0, st>>>(L.ds, L.es, nc);
    k_lifted_add<<<grid_of(nc), LBS, 0, st>>>(L.dl, L.el, nc);
    ++k;
  }
  if (sweeps) *sweeps = k;
  if (relp) *relp = rel;
  if (!std::isfinite(rel)) { set_error("non-finite lifted solution"); return COLLO_ERR_NUMERIC; }
  return COLLO_OK;
}

}  // namespace collo

extern "C" {

collo_status collo_lifted_factor(collo_problem* prob, const double* sigma_x, const double* sigma_s,
                                 double delta_w, int* positive_definite) {
  if (!prob || !sigma_s) { set_error("NULL argument"); return COLLO_ERR_INVALID_ARG; }
  if (!prob->evaluated) { set_error("collo_eval has not run"); return COLLO_ERR_NOT_EVALUATED; }
  if (!std::isfinite(delta_w) || delta_w < 0) {
    set_error("delta_w must be finite and >= 0"); return COLLO_ERR_INVALID_ARG;
  }
  COLLO_CUDA(cudaSetDevice(prob->device));
  collo_status s = lifted_storage(prob);
  if (s != COLLO_OK) return s;
  DevLifted& L = prob->lifted->V;
  cudaStream_t st = prob->stream;
  const size_t nx = prob->n_x, nc = prob->n_c;
  prob->lifted->pd = false;
  prob->lifted->eval_count = -1;
  if (sigma_x)
    COLLO_CUDA(cudaMemcpyAsync(L.sigx, sigma_x, nx * sizeof(double), cudaMemcpyDefault, st));
  else
    COLLO_CUDA(cudaMemsetAsync(L.sigx, 0, nx * sizeof(double), st));
  COLLO_CUDA(cudaMemcpyAsync(L.d, sigma_s, nc * sizeof(double), cudaMemcpyDefault, st));
  bool pd = false;
  if ((s = lifted_factor_dev(prob, L.d, delta_w, &pd)) != COLLO_OK) return s;
  if (positive_definite) *positive_definite = pd ? 1 : 0;
  return COLLO_OK;
}

collo_status collo_lifted_solve(collo_problem* prob, const double* r_x, const double* r_s,
                                const double* r_c, double* dx, double* ds, double* dlam,
                                int refine_max, double refine_tol, collo_solve_info* info) {
  if (!prob || !r_x || !r_s || !r_c || !dx || !ds || !dlam) {
    set_error("NULL argument"); return COLLO_ERR_INVALID_ARG;
  }
  if (!prob->lifted || !prob->lifted->pd || prob->lifted->eval_count != prob->eval_count) {
    set_error("no positive definite lifted factorization of the current evaluation");
    return COLLO_ERR_NOT_FACTORED;
  }
  COLLO_CUDA(cudaSetDevice(prob->device));
  DevLifted& L = prob->lifted->V;
  cudaStream_t st = prob->stream;
  const size_t nx = prob->n_x, nc = prob->n_c;
  COLLO_CUDA(cudaMemcpyAsync(L.rx, r_x, nx * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(cudaMemcpyAsync(L.rs, r_s, nc * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(cudaMemcpyAsync(L.rc, r_c, nc * sizeof(double), cudaMemcpyDefault, st));
  int k = 0;
  double rel = 0.0;
  collo_status s = lifted_solve_dev(prob, refine_max, refine_tol, &k, &rel);
  if (info) { info->refinement_sweeps = k; info->residual = rel; }
  if (s != COLLO_OK) return s;
  COLLO_CUDA(cudaMemcpyAsync(dx, L.dx, nx * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(cudaMemcpyAsync(ds, L.ds, nc * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(cudaMemcpyAsync(dlam, L.dl, nc * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  return COLLO_OK;
}

}  // extern "C"
