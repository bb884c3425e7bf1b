// Structured, pivot-free factorization and solve of the element-banded KKT
// system bordered by the parameter block.
//
// The paper attributes most of the GPU benefit to sparse linear algebra on a
// KKT system put in a "pivoting-free factorizable form", with parallelism at
// the level of the elimination tree (Abstract; Introduction).  Here the
// elimination tree is explicit:
//
//  1. Element condensation (one CUDA block per element, all elements in
//     parallel): the element's 8n unknowns are ordered as n (state,
//     multiplier) pairs per group -- (z1,c1), (z2,c2), (z0,c3) interior and
//     (z3,c0) interface -- and the 3n interior pairs are eliminated with
//     static 2x2 pivots [[w, j], [j, -delta_c]].  Their determinant is
//     -(w delta_c + j^2) < 0 for the collocation Jacobian entry j, so each pivot
//     is nonsingular whatever the sign of the Hessian entry w; the sequence is
//     Gaussian elimination without pivoting on the element's square
//     collocation Jacobian.  The parameter border rides along as extra rows.
//  2. Block cyclic reduction over the chain of 2n x 2n interface blocks
//     (ceil(log2 N) levels; at each level the odd blocks are eliminated in
//     parallel, each updating its two neighbours, creating the n x n fill
//     coupling between them, and contributing to the parameter Schur block).
//  3. The p x p parameter Schur complement, summed from all contributions in
//     a fixed order and factored in FP64 (LDL^T, 1x1 pivots).
//
// Inertia is counted from every pivot block (Sylvester's law of inertia).
// T = double (plain path) or float (mixed path; residuals and refinement
// are FP64 elsewhere).
#include <map>
#include <mutex>
#include <tuple>

#include "collo_internal.cuh"

namespace collo {

constexpr int FBS = 256;   // threads per factor block
constexpr int FTY = FBS / 32;

__device__ inline void pivot_inertia(double a, double b, double d, int& pos, int& neg, int& zero) {
  const double det = fma(a, d, -(b * b));
  if (!(det == det) || det == 0.0 || !isfinite(det)) { zero += 2; return; }
  if (det < 0) { pos += 1; neg += 1; return; }
  if (a + d > 0) pos += 2; else neg += 2;
}

// Packed lower triangle: entry (r, c), c <= r, at r (r + 1) / 2 + c.
__host__ __device__ inline int tri_at(int r, int c) { return r * (r + 1) / 2 + c; }

// Tile t of a lower triangle of tiles, numbered row by row: (ti, tj), tj <= ti.
__device__ inline void tri_tile(int t, int& ti, int& tj) {
  int i = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  ti = i;
  tj = t - i * (i + 1) / 2;
}

// Panel buffer leading dimension: odd (the per-row and per-column accesses of
// the panel eliminations spread over the banks) and PANEL_PAD rows past msz, so
// that every warp tile of trailing_update (rows below msz + 4 TR, columns below
// msz + 4 TR + 8 TC) reads inside the buffer.
constexpr int PANEL_PAD = 96;
__host__ __device__ inline int panel_ld(int msz) { return (msz + PANEL_PAD) | 1; }

// Trailing update of pair_eliminate_packed for kernels with a small register
// budget (the cyclic-reduction blocks inside the cooperative factorization
// kernel when it runs three blocks per SM): 4 x 4 tiles of the packed
// triangle, one per thread at a time; A[r][c] -= (sum_k Lp[k][r] W[k][c]), the
// sum in ascending k, subtracted once (the same arithmetic per entry as
// trailing_update, so the result does not depend on which of the two a
// launch uses).
template <typename T>
__device__ void trailing_update_tiles4(T* A, int msz, int cend, int K, const T* __restrict__ Lp,
                                       const T* __restrict__ W, int ldw) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int Tn = msz - cend;
  if (Tn > 0) {
    const int ntr = (Tn + 3) >> 2;
    const int ntiles = ntr * (ntr + 1) / 2;
    for (int t = tid; t < ntiles; t += nt) {
      int ti, tj;
      tri_tile(t, ti, tj);
      const int r0 = cend + 4 * ti, cb = cend + 4 * tj;
      // the tile's entries are loaded first, so that their latency (the
      // triangle may be in global memory) overlaps the products below
      T cur[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int r = r0 + u, c = cb + v;
          cur[u][v] = (r < msz && c <= r) ? A[tri_at(r, c)] : T(0);
        }
      T acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
      for (int k = 0; k < K; ++k) {
        T lr[4], uc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          lr[u] = (r0 + u < msz) ? Lp[k * ldw + r0 + u] : T(0);
          uc[u] = (cb + u < msz) ? W[k * ldw + cb + u] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fma(lr[u], uc[v], acc[u][v]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + u;
        if (r >= msz) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int c = cb + v;
          if (c <= r) A[tri_at(r, c)] = cur[u][v] - acc[u][v];
        }
      }
    }
  }
}

// Trailing update of pair_eliminate_packed: A[r][c] -= sum_k Lp[k][r] W[k][c]
// for cend <= c <= r < msz (packed lower triangle, shared or global memory),
// the sum over k = 0..K-1 in ascending order, subtracted once.  Warp-blocked
// register tiles: a warp owns 4 TR rows x 8 TC columns of the trailing
// matrix, lane (ty, tx) = (lane / 8, lane % 8) the rows r0 + ty + 4u (u < TR)
// and the columns c0 + tx + 8v (v < TC), so that for every k the warp reads
// 4 TR entries of Lp[k] in runs of 4 and 8 TC entries of W[k] in runs of 8
// (no bank conflicts), and each thread does TR TC multiply-adds per TR + TC
// shared loads at fixed offsets from one address per k.  TR x TC is set by
// the register budget of the calling kernel; out of line, so that the tile
// gets the kernel's whole register budget.  Rows and columns past msz are
// computed from the panel buffers' padding and never stored.
template <typename T, int TR, int TC>
__device__ __noinline__ void trailing_update(T* A, int msz, int cend, int K,
                                             const T* __restrict__ Lp, const T* __restrict__ W,
                                             int ldw) {
  constexpr int WR = 4 * TR, WC = 8 * TC;
  static_assert(WR + WC <= PANEL_PAD, "panel buffers padded for the warp tile");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ty = lane >> 3, tx = lane & 7;
  const int Tn = msz - cend;
  if (Tn <= 0) return;
  const int nbr = (Tn + WR - 1) / WR;
  int blk = 0;
  for (int bi = 0; bi < nbr; ++bi) {
    const int nbc = ((bi + 1) * WR + WC - 1) / WC;   // blocks meeting the lower triangle
    for (int bj = 0; bj < nbc; ++bj, ++blk) {
      if (blk % nw != warp) continue;
      const int r0 = cend + bi * WR + ty, c0 = cend + bj * WC + tx;
      // rows / columns past msz (fewer than WR + WC) read the padding of the
      // panel buffers: indeterminate values in entries never stored
      const T* lb = Lp + r0;
      const T* wb = W + c0;
      // the tile's entries are loaded first, so that their latency (the
      // triangle may be in global memory) overlaps the products
      T cur[TR][TC], acc[TR][TC];
#pragma unroll
      for (int u = 0; u < TR; ++u)
#pragma unroll
        for (int v = 0; v < TC; ++v) {
          const int r = r0 + 4 * u, c = c0 + 8 * v;
          cur[u][v] = (r < msz && c <= r) ? A[tri_at(r, c)] : T(0);
          acc[u][v] = T(0);
        }
#pragma unroll 2
      for (int k = 0; k < K; ++k) {
        const T* lk = lb + k * ldw;
        const T* wk = wb + k * ldw;
        T lr[TR], uc[TC];
#pragma unroll
        for (int u = 0; u < TR; ++u) lr[u] = lk[4 * u];
#pragma unroll
        for (int v = 0; v < TC; ++v) uc[v] = wk[8 * v];
#pragma unroll
        for (int u = 0; u < TR; ++u)
#pragma unroll
          for (int v = 0; v < TC; ++v) acc[u][v] = fma(lr[u], uc[v], acc[u][v]);
      }
#pragma unroll
      for (int u = 0; u < TR; ++u) {
        const int r = r0 + 4 * u;
        if (r >= msz) continue;
#pragma unroll
        for (int v = 0; v < TC; ++v) {
          const int c = c0 + 8 * v;
          if (c <= r) A[tri_at(r, c)] = cur[u][v] - acc[u][v];
        }
      }
    }
  }
}


// Eliminate the first npairs (state, multiplier) pairs of the symmetric msz x
// msz matrix A, stored as a packed lower triangle (shared or global memory),
// blocked right-looking: pairs are taken in panels of PB.  A panel's 2 PB
// columns (rows >= the panel) are copied into W[j][r] (leading dimension
// ldw = panel_ld(msz)).  One warp eliminates the panel's pairs on its own 2 PB rows
// (the diagonal block), recording each pair's pivot inverse; then every
// thread replays the same eliminations on the rows below, one row at a time
// in registers (a row's multipliers depend only on the diagonal block), with
// no barrier between pairs; then the trailing matrix receives one rank-2PB
// update, in register tiles of TR x TC (4 x 4 per thread at a time for TR = 0),
// from the multipliers Lp[j][r] and the unscaled columns W.  Every entry sees the arithmetic, in the order, of the
// pair-by-pair elimination: the pivot inverse ia = d / det, ib = -b / det,
// id = a / det; multipliers l0 = x0 ia + x1 ib, l1 = x0 ib + x1 id; the
// panel's remaining columns updated pair by pair; trailing entries by the sum
// over the panel's 2 PB columns in ascending order, subtracted once
// (trailing_update for TR x TC > 0, trailing_update_tiles4 for TR = 0).
// L columns go to Lout[c * lds + r] (rows r > pair), pivots (a, b, d) to
// Dout[3 q]; pivot inertia is counted by thread 0.  The trailing block (rows
// and columns >= 2 npairs) is left in A.
// PB is 8 for blocks held in shared memory and 16 for blocks in the global
// slab (half the trailing passes over global memory, twice the arithmetic per
// entry read and written).
template <typename T, int PB, int TR, int TC>
__device__ void pair_eliminate_packed(T* A, int msz, int npairs, T* __restrict__ Lout, int lds,
                                      T* __restrict__ Dout, T* Lp, T* W, int& pos, int& neg,
                                      int& zero) {
  const int tid = threadIdx.x, nt = blockDim.x, ldw = panel_ld(msz);
  __shared__ T pinv[PB][3];   // pivot inverse (ia, ib, id) of the panel's pairs
  for (int q0 = 0; q0 < npairs; q0 += PB) {
    const int pe = min(q0 + PB, npairs);
    const int cp = 2 * q0, cend = 2 * pe, K = cend - cp, rows = msz - cp;
    // panel columns cp .. cend-1 for rows >= cp (the lower triangle; the
    // entries above the diagonal are never read)
    for (int idx = tid; idx < K * rows; idx += nt) {
      const int r = cp + idx / K, j = idx - (r - cp) * K, c = cp + j;
      if (c <= r) W[j * ldw + r] = A[tri_at(r, c)];
    }
    __syncthreads();
    // 1. the diagonal block (rows cp .. cend-1), pair by pair, by warp 0
    if (tid < 32) {
      const int lane = tid;
      for (int q = q0; q < pe; ++q) {
        const int c0 = 2 * q, c1 = c0 + 1, kk = 2 * (q - q0);
        const T a = W[kk * ldw + c0], b = W[kk * ldw + c1], d = W[(kk + 1) * ldw + c1];
        const T det = fma(a, d, -(b * b));
        T ia, ib, id;
        if (det != T(0) && isfinite(det)) {
          const T inv = T(1) / det;
          ia = d * inv; ib = -b * inv; id = a * inv;
        } else {
          ia = ib = id = T(0);
        }
        if (lane == 0) {
          Dout[3 * q + 0] = a; Dout[3 * q + 1] = b; Dout[3 * q + 2] = d;
          pinv[q - q0][0] = ia; pinv[q - q0][1] = ib; pinv[q - q0][2] = id;
          pivot_inertia((double)a, (double)b, (double)d, pos, neg, zero);
        }
        const int r = c1 + 1 + lane;
        if (r < cend) {
          const T x0 = W[kk * ldw + r], x1 = W[(kk + 1) * ldw + r];
          const T l0 = fma(x0, ia, x1 * ib);
          const T l1 = fma(x0, ib, x1 * id);
          Lout[(size_t)c0 * lds + r] = l0;
          Lout[(size_t)c1 * lds + r] = l1;
          for (int c = c1 + 1; c <= r; ++c) {   // remaining panel columns, c <= r
            T& w = W[(c - cp) * ldw + r];
            w = fma(-l1, W[(kk + 1) * ldw + c], fma(-l0, W[kk * ldw + c], w));
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // 2. rows below the panel: the same eliminations, each thread on its own
    // rows (entries of row r are updated in place in W; the diagonal block's
    // columns are read through a volatile view, loaded where used)
    const volatile T* U = W;
    for (int r = cend + tid; r < msz; r += nt) {
      for (int kk = 0; kk < K; kk += 2) {
        const T ia = pinv[kk >> 1][0], ib = pinv[kk >> 1][1], id = pinv[kk >> 1][2];
        const T x0 = W[kk * ldw + r], x1 = W[(kk + 1) * ldw + r];
        const T l0 = fma(x0, ia, x1 * ib);
        const T l1 = fma(x0, ib, x1 * id);
        Lp[kk * ldw + r] = l0;
        Lp[(kk + 1) * ldw + r] = l1;
        Lout[(size_t)(cp + kk) * lds + r] = l0;
        Lout[(size_t)(cp + kk + 1) * lds + r] = l1;
        for (int j = kk + 2; j < K; ++j) {
          const int c = cp + j;
          T& w = W[j * ldw + r];
          w = fma(-l1, U[(kk + 1) * ldw + c], fma(-l0, U[kk * ldw + c], w));
        }
      }
    }
    __syncthreads();
    // trailing rank-K update of rows / columns >= cend (lower part)
    if constexpr (TR == 0)
      trailing_update_tiles4<T>(A, msz, cend, K, Lp, W, ldw);
    else
      trailing_update<T, TR, TC>(A, msz, cend, K, Lp, W, ldw);
    __syncthreads();
  }
}

// Storage of a block of msz rows factored by pair_eliminate_packed: the two
// panel buffers Lp, W (2 PB x panel_ld(msz) each) and the packed triangle
// (msz (msz + 1) / 2).  Everything in shared memory (PB = 8) when it fits the
// factorization limit; otherwise (PB = 16) the triangle in a per-CUDA-block
// global slab (L2-resident) and the panel buffers in shared memory, or, when
// even they do not fit, in the slab behind the triangle.
__host__ __device__ inline size_t big_tri_elems(int msz) {
  return ((size_t)msz * (msz + 1) / 2 + 1) & ~size_t(1);
}
template <typename T>
__host__ __device__ inline int big_pb(int msz) {
  const size_t full8 = sizeof(T) * (2 * (size_t)16 * panel_ld(msz) + big_tri_elems(msz));
  return full8 <= FACTOR_SMEM_LIMIT ? 8 : 16;
}
template <typename T>
__host__ __device__ inline size_t big_panel_elems(int msz) {
  return 2 * (size_t)(2 * big_pb<T>(msz)) * panel_ld(msz);
}
// pair_eliminate_packed with PB = pb (8, or 16 for a block in the global slab,
// whose panel buffers are sized for 16)
template <typename T, int TR, int TC>
__device__ inline void pair_eliminate_big(T* A, int msz, int npairs, T* __restrict__ Lout,
                                          int lds, T* __restrict__ Dout, T* Lp, T* W, int& pos,
                                          int& neg, int& zero, int pb) {
  if (pb == 16)
    pair_eliminate_packed<T, 16, TR, TC>(A, msz, npairs, Lout, lds, Dout, Lp, W, pos, neg, zero);
  else
    pair_eliminate_packed<T, 8, TR, TC>(A, msz, npairs, Lout, lds, Dout, Lp, W, pos, neg, zero);
}
template <typename T>
__host__ __device__ inline bool panel_in_global(int msz) {
  return sizeof(T) * big_panel_elems<T>(msz) > FACTOR_SMEM_LIMIT;
}
template <typename T>
__host__ __device__ inline size_t slab_elems(int msz) {
  return big_tri_elems(msz) + (panel_in_global<T>(msz) ? big_panel_elems<T>(msz) : 0);
}
template <typename T>
struct BigPlace {
  T* A;
  T* Lp;
  T* W;
};
// Pointers of block storage for this CUDA block (full: all in shared memory).
template <typename T>
__device__ inline BigPlace<T> big_place(unsigned char* smraw, T* work, int msz, bool full) {
  const size_t pn = big_panel_elems<T>(msz) / 2;
  T* slab = work + (size_t)blockIdx.x * slab_elems<T>(msz);
  const bool pg = !full && panel_in_global<T>(msz);
  T* Lp = pg ? slab + big_tri_elems(msz) : reinterpret_cast<T*>(smraw);
  T* A = full ? Lp + 2 * pn : slab;
  return {A, Lp, Lp + pn};
}

// Scatter assembly of element e's KKT block (packed lower triangle blk, zeroed)
// from its FP64 derivative blocks Wzz, JZ (K n^2), Wzt, JT (K n p), Wobj
// ((K+1)^2 n) and the barrier diagonal sig ((K+1) n, or NULL: zero), which may be in
// shared or global memory.  Out of line (it is not on the elimination's
// path).  Three passes separated by barriers over the nt
// threads of the block: disjoint entries (point Hessian blocks, the identity
// parts of the collocation rows D[k][j], continuity / initial rows, -delta_c,
// border), sums onto those (objective blocks, -h df/dz), then the diagonal.
template <typename T>
__device__ __noinline__ void elem_scatter(const DevProb& P, int e, const double* Wzz,
                                          const double* JZ, const double* Wzt, const double* JT,
                                          const double* Wobj, const double* sig, double dw,
                                          double dc, T* blk);
template <typename T, class Tr>
__device__ __noinline__ void gauss_chain_out(const DevProb& P, const DevFactor<T>& F, int e,
                                             int i0, double dc, Tr tr);

// ---- 1. element condensation --------------------------------------------------
// One CUDA block condenses element e: assemble the bordered (2 (K+1) n + p)
// block, eliminate the K n interior pairs, write L, pivots, the 2n x 2n chain
// block, its border, the p x p Schur contribution and the coupling (Radau:
// -I; Gauss: gauss_chain_out).  For blocks above the register-tile limit
// (elem_factor_rt below).  TR x TC: the trailing update's register tile
// (trailing_update), set by the calling kernel's register budget.
template <typename T, int TR, int TC>
__device__ void elem_factor_big(const DevProb& P, const DevEval& E,
                                const double* __restrict__ sigma, double dw, double dc,
                                const DevFactor<T>& F, int e, const BigPlace<T>& pl, int pb) {
  const int n = P.n, p = P.p, m = P.m, ext = P.ext, K = P.K, npt = P.np;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nint = K * n;          // interior pairs
  const int i0 = 2 * nint;         // first chain row (2Kn)
  const size_t nn = (size_t)n * n, np = (size_t)n * p;
  T* A = pl.A;
  const int ntri = ext * (ext + 1) / 2;
  for (int i = tid; i < ntri; i += nt) A[i] = T(0);
  __syncthreads();
  elem_scatter<T>(P, e, E.Wzz + (size_t)e * K * nn, E.JZ + (size_t)e * K * nn,
                  E.Wzt + (size_t)e * K * np, E.JT + (size_t)e * K * np,
                  E.Wobj + (size_t)e * npt * npt * n,
                  sigma ? sigma + (size_t)e * npt * n : nullptr, dw, dc, A);
  int pos = 0, neg = 0, zero = 0;
  pair_eliminate_big<T, TR, TC>(A, ext, nint, F.Lel + (size_t)e * (2 * nint) * ext, ext,
                        F.Del + (size_t)e * nint * 3, pl.Lp, pl.W, pos, neg, zero, pb);
  if (tid == 0) {
    F.inert[e * 3 + 0] = pos; F.inert[e * 3 + 1] = neg; F.inert[e * 3 + 2] = zero;
  }
  const int n2 = 2 * n;
  auto tr = [&](int a, int b) { return a >= b ? A[tri_at(a, b)] : A[tri_at(b, a)]; };
  double* Sc = F.Scon + (size_t)e * p * p;
  for (int idx = tid; idx < p * p; idx += nt) {
    const int q = idx / p, q2 = idx - q * p;
    Sc[idx] = (double)tr(m + q, m + q2);
  }
  if (P.gauss) {
    gauss_chain_out<T>(P, F, e, i0, dc, tr);
    __syncthreads();
    return;
  }
  T* Aif = F.Aif + (size_t)e * n2 * n2;
  for (int idx = tid; idx < n2 * n2; idx += nt) {
    const int u = idx / n2, v = idx - u * n2;
    Aif[idx] = tr(i0 + u, i0 + v);
  }
  T* Bif = F.Bif + (size_t)e * n2 * p;
  for (int idx = tid; idx < n2 * p; idx += nt) {
    const int u = idx / p, q = idx - u * p;
    Bif[idx] = A[tri_at(m + q, i0 + u)];
  }
  T* C = F.Cpl + (size_t)e * n * n;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int s2 = idx / n, t = idx - s2 * n;
    C[idx] = (!chain_start(P, e) && s2 == t) ? T(-1) : T(0);
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(FBS)
k_elem_factor(DevProb P, DevEval E, const double* __restrict__ sigma, double dw, double dc,
              DevFactor<T> F, int use_smem, int slab_pb) {
  extern __shared__ unsigned char smraw[];
  const BigPlace<T> pl = big_place<T>(smraw, F.work, P.ext, use_smem != 0);
  for (int e = blockIdx.x; e < P.N; e += gridDim.x)
    elem_factor_big<T, 8, sizeof(T) == 4 ? 8 : 4>(P, E, sigma, dw, dc, F, e, pl,
                                                  use_smem ? 8 : slab_pb);
}

// ---- 1'. pair elimination with the block held in registers -------------------------
// The same elimination as pair_eliminate, organised for small blocks
// (ext <= RT_MAX_EXT): the lower triangle is cut into 4 x 4 tiles and each of
// the NT threads keeps up to TPT tiles in registers for the whole
// elimination.  For every pair the owners of the pair's tile column publish
// the two pivot columns (rows >= the pair) into a shared vector; after one
// barrier every thread forms the pivot inverse and the multipliers of its own
// rows and applies the rank-2 update to its tiles.  The shared vector
// alternates between two buffers, so one barrier per pair suffices: a buffer
// is rewritten only after the barrier that follows all reads of it.  Entries
// that are already eliminated, above the diagonal or past ext take harmless
// finite updates and are never read again.
//   entry(r, c), c <= r < ext: the block's lower triangle (assembly);
//   sink(r, c, v), 2 npairs <= c <= r < ext: the eliminated trailing block;
//   bar(): barrier over the NT threads; tid in [0, NT).
// L columns go to Lout[c * lds + r] (rows r > pair), pivots (a, b, d) to
// Dout[3 q] and pivs[q] (recorded by thread 0, in PAIRED mode by the owner of
// the diagonal tile); after the loop the threads count the pivots' inertia
// into cnt[0..2].  In PAIRED mode the loop's barrier is named barrier 1 over
// the warps that still have work (below); bar() is used outside the loop.
constexpr int RT_MAX_TR = 31;            // tile rows: ext <= 124
constexpr int RT_UB = 4 * RT_MAX_TR + 4;  // rows per pivot-column buffer

template <typename T>
struct alignas(2 * sizeof(T)) Pair {
  T x, y;
};
// Pivot-column buffers: two per elimination, 16-byte aligned for load4.
template <typename T>
struct alignas(16) PivotBuf {
  Pair<T> v[2 * RT_UB];
};

// Four consecutive entries of a pivot-column buffer (16-byte aligned).
__device__ inline void load4(const Pair<float>* p, float x[4], float y[4]) {
  const float4 u = reinterpret_cast<const float4*>(p)[0];
  const float4 v = reinterpret_cast<const float4*>(p)[1];
  x[0] = u.x; y[0] = u.y; x[1] = u.z; y[1] = u.w;
  x[2] = v.x; y[2] = v.y; x[3] = v.z; y[3] = v.w;
}
__device__ inline void load4(const Pair<double>* p, double x[4], double y[4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const double2 w = reinterpret_cast<const double2*>(p)[u];
    x[u] = w.x; y[u] = w.y;
  }
}

template <typename T>
struct Pivot {
  T a, b, d;
};
// Correctly rounded reciprocal (the same value as 1 / x).
__device__ inline float recip_rn(float x) { return __frcp_rn(x); }
__device__ inline double recip_rn(double x) { return __drcp_rn(x); }

// Asynchronous copies (cp.async, completed by cp_async_wait_all) of single
// elements from global to shared memory.
template <typename T>
__device__ inline void cp_async_elem(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
constexpr int RT_MAX_PAIRS = 2 * RT_MAX_TR + 2;   // pairs of a block of <= 124 rows
constexpr int RT_MAX_THREADS = 512;               // threads of a register-tiled block

// Tiles are owned in pairs along a tile row: pair (ti, k) is tiles (ti, 2k) and
// (ti, 2k + 1) (the second absent when 2k + 1 > ti), so the multipliers of the
// row are formed once for both.  Pairs are numbered column pair by column pair
// (k ascending, then ti from 2k to R - 1; R - 2k pairs in column pair k), so
// that the threads of a warp hold neighbouring column pairs and finish
// together: a pair has no work left after pair step 4k + 1 (one tile) or
// 4k + 3 (two tiles), when its columns are eliminated and published.
__host__ __device__ inline int tile_pairs(int R) { return (R + 1) * (R + 1) / 4; }
__device__ inline void tile_pair(int t, int R, int& ti, int& k) {
  // first pair of column pair k: k (R + 1 - k)
  int c = (int)(0.5f * ((float)(R + 1) - sqrtf((float)((R + 1) * (R + 1) - 4 * t))));
  if (c < 0) c = 0;
  while (c > 0 && c * (R + 1 - c) > t) --c;
  while ((c + 1) * (R - c) <= t) ++c;
  k = c;
  ti = 2 * c + (t - c * (R + 1 - c));
}

// PAIRED: each thread owns TPP row pairs of tiles (above); otherwise TPP
// single tiles (for latency-bound small blocks, where every thread should
// hold a tile).
template <typename T, int TPP, bool PAIRED, class Entry, class Sink, class Bar>
__device__ void pair_eliminate_rt(int tid, int nt, int ext, int npairs, Entry entry,
                                  T* __restrict__ Lout, int lds, T* __restrict__ Dout, Sink sink,
                                  Bar bar, Pair<T>* ub, Pivot<T>* pivs, int* cnt) {
  constexpr int H = PAIRED ? 2 : 1;
  const int R = (ext + 3) >> 2, npr = PAIRED ? tile_pairs(R) : R * (R + 1) / 2;
  for (int r = tid; r < 2 * RT_UB; r += nt) ub[r] = Pair<T>{T(0), T(0)};
  int ti[TPP], tj0[TPP];
  bool two[TPP];
  T a[TPP][H][4][4];
#pragma unroll
  for (int j = 0; j < TPP; ++j) {
    const int t = tid + nt * j;
    int k = 0;
    ti[j] = -1;
    if (PAIRED) {
      if (t < npr) tile_pair(t, R, ti[j], k);
      tj0[j] = 2 * k;
      two[j] = tj0[j] + 1 <= ti[j];
    } else {
      tj0[j] = 0;
      if (t < npr) tri_tile(t, ti[j], tj0[j]);
      two[j] = false;
    }
#pragma unroll
    for (int h = 0; h < H; ++h)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int r = 4 * ti[j] + u, c = 4 * (tj0[j] + h) + v;
          a[j][h][u][v] = (ti[j] >= 0 && (h == 0 || two[j]) && r < ext && c <= r) ? entry(r, c)
                                                                                  : T(0);
        }
  }
  // PAIRED: a warp leaves the pair loop once none of its threads has work left
  // (exit pair = max over its threads of 4k + 2 or 4k + 4); the loop's barrier
  // (named barrier 1) of pair q counts the warps whose exit pair is >= q: those
  // still working wait on it, the one leaving at q only arrives, so its reads
  // of the previous pivot buffer are ordered before that buffer is rewritten.
  int* s_exit = nullptr;
  int* s_count = nullptr;
  int my_exit = npairs;
  if constexpr (PAIRED) {
    __shared__ int exit_of_warp[RT_MAX_THREADS / 32];
    __shared__ int count_of_pair[RT_MAX_PAIRS];
    s_exit = exit_of_warp;
    s_count = count_of_pair;
    int qd = 0;
#pragma unroll
    for (int j = 0; j < TPP; ++j)
      if (ti[j] >= 0) qd = max(qd, min(npairs, two[j] ? 2 * tj0[j] + 4 : 2 * tj0[j] + 2));
    qd = (int)__reduce_max_sync(0xffffffffu, (unsigned)qd);
    if ((tid & 31) == 0) s_exit[tid >> 5] = qd;
  }
  bar();
  if constexpr (PAIRED) {
    const int nw = nt >> 5;
    for (int q = tid; q < npairs; q += nt) {
      int c = 0;
      for (int w = 0; w < nw; ++w) c += s_exit[w] >= q ? 32 : 0;
      s_count[q] = c;
    }
    my_exit = s_exit[tid >> 5];
    bar();
  }
  for (int q = 0; q < npairs; ++q) {
    if constexpr (PAIRED) {
      if (q >= my_exit) {
        asm volatile("bar.arrive 1, %0;" ::"r"(s_count[q]) : "memory");
        break;
      }
    }
    const int c0 = 2 * q, c1 = c0 + 1, tq = c0 >> 2;
    const bool hi = (c0 & 2) != 0;
    Pair<T>* b = ub + (q & 1) * RT_UB;
#pragma unroll
    for (int j = 0; j < TPP; ++j)
#pragma unroll
      for (int h = 0; h < H; ++h)
        if (ti[j] >= 0 && tj0[j] + h == tq && (h == 0 || two[j]))
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = 4 * ti[j] + u;
            if (r >= c0 && r < ext)
              b[r] = Pair<T>{hi ? a[j][h][u][2] : a[j][h][u][0], hi ? a[j][h][u][3] : a[j][h][u][1]};
          }
    if constexpr (PAIRED) asm volatile("bar.sync 1, %0;" ::"r"(s_count[q]) : "memory");
    else bar();
    const T pa = b[c0].x, pb = b[c1].x, pd = b[c1].y;
    const T det = fma(pa, pd, -(pb * pb));
    T ia, ib, id;
    if (det != T(0) && isfinite(det)) {
      const T inv = recip_rn(det);
      ia = pd * inv; ib = -pb * inv; id = pa * inv;
    } else {
      ia = ib = id = T(0);
    }
    // the pivots are recorded by thread 0, or in PAIRED mode by the owner of the
    // diagonal tile (tq, tq), which works at this step
    bool writer = tid == 0;
    if constexpr (PAIRED) {
      writer = false;
#pragma unroll
      for (int j = 0; j < TPP; ++j)
        writer = writer || (ti[j] == tq && (tj0[j] == tq || (two[j] && tj0[j] + 1 == tq)));
    }
    if (writer) {
      Dout[3 * q + 0] = pa; Dout[3 * q + 1] = pb; Dout[3 * q + 2] = pd;
      pivs[q] = Pivot<T>{pa, pb, pd};
    }
#pragma unroll
    for (int j = 0; j < TPP; ++j) {
      if (ti[j] < 0 || 4 * ti[j] + 3 <= c1) continue;   // no live row
      T l0[4], l1[4], xr0[4], xr1[4];
      load4(b + 4 * ti[j], xr0, xr1);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        l0[u] = fma(xr0[u], ia, xr1[u] * ib);
        l1[u] = fma(xr0[u], ib, xr1[u] * id);
      }
      if (tj0[j] == tq || (two[j] && tj0[j] + 1 == tq))
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = 4 * ti[j] + u;
          if (r > c1 && r < ext) {
            Lout[(size_t)c0 * lds + r] = l0[u];
            Lout[(size_t)c1 * lds + r] = l1[u];
          }
        }
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int tj = tj0[j] + h;
        if ((h == 1 && !two[j]) || 4 * tj + 3 <= c1) continue;   // no live column
        T y0[4], y1[4];
        load4(b + 4 * tj, y0, y1);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v)
            a[j][h][u][v] = fma(-l1[u], y1[v], fma(-l0[u], y0[v], a[j][h][u][v]));
      }
    }
  }
  const int cs = 2 * npairs;
#pragma unroll
  for (int j = 0; j < TPP; ++j) {
    if (ti[j] < 0) continue;
#pragma unroll
    for (int h = 0; h < H; ++h) {
      if (h == 1 && !two[j]) continue;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int r = 4 * ti[j] + u, c = 4 * (tj0[j] + h) + v;
          if (r < ext && c <= r && c >= cs) sink(r, c, a[j][h][u][v]);
        }
    }
  }
  // inertia of the pivots (exact FP64 sign test), off the elimination's
  // critical path: cnt[0..2] = (pos, neg, zero) after the final barrier
  if (tid < 3) cnt[tid] = 0;
  bar();
  int pos = 0, neg = 0, zero = 0;
  for (int q = tid; q < npairs; q += nt)
    pivot_inertia((double)pivs[q].a, (double)pivs[q].b, (double)pivs[q].d, pos, neg, zero);
  if (pos) atomicAdd(&cnt[0], pos);
  if (neg) atomicAdd(&cnt[1], neg);
  if (zero) atomicAdd(&cnt[2], zero);
  bar();
}

struct CtaBar {
  __device__ void operator()() const { __syncthreads(); }
};
// Barrier over the 128 threads of one half of a 256-thread block (named
// barrier 1 + half; barrier 0 is __syncthreads).
struct HalfBar {
  int id;
  __device__ void operator()() const {
    if (id == 1) asm volatile("bar.sync 1, 128;" ::: "memory");
    else asm volatile("bar.sync 2, 128;" ::: "memory");
  }
};

// Element block of elem_factor_rt, assembled in shared memory as a packed
// lower triangle (entry (r, c), c <= r, at r (r + 1) / 2 + c) by structured
// scatter passes over the element's derivative blocks, then loaded into the
// threads' register tiles; after the elimination the trailing blocks go back
// through the same buffer and leave in coalesced stores.
template <typename T>
__host__ __device__ inline size_t elem_blk_bytes(const DevProb& P) {
  return (sizeof(T) * ((size_t)P.ext * (P.ext + 1) / 2) + 15) & ~size_t(15);
}
// The element's FP64 derivative blocks (Wzz, JZ: K n^2 each; Wzt, JT: K n p
// each; Wobj: (K+1)^2 n; sigma: (K+1) n), staged behind the triangle.
__host__ __device__ inline size_t elem_raw_doubles(const DevProb& P) {
  const size_t K = P.K, np = P.np;
  return 2 * K * P.n * P.n + 2 * K * P.n * P.p + (np * np + np) * P.n;
}
template <typename T>
__host__ __device__ inline size_t elem_stage_bytes(const DevProb& P) {
  return elem_blk_bytes<T>(P) + sizeof(double) * elem_raw_doubles(P);
}
// i / d and i % d for 0 <= i < 2^22 and 1 <= d <= 4096 through the float
// reciprocal inv = 1 / d: (i + 0.5) / d lies at least 0.5 / d from an integer,
// far more than the float rounding of the product, so the truncation is exact.
__device__ inline int quot(int i, int d, float inv) {
  return (int)(((float)i + 0.5f) * inv);
}
// local index of the state of point j / the multiplier of the element's
// constraint k (groups of grp_point / grp_con): Radau (z1,c1), (z2,c2),
// (z0,c3), (z3,c0); Gauss (z1,c1) .. (z4,c4), (z0, c0 of the next element),
// whose multiplier is k = 0 here
__device__ inline int loc_state(const DevProb& P, int j, int s) {
  const int K = P.K;
  const int g = j == 0 ? (P.gauss ? K : K - 1) : ((!P.gauss && j == K) ? K : j - 1);
  return 2 * (g * P.n + s);
}
__device__ inline int loc_dual(const DevProb& P, int k, int s) {
  return 2 * ((k == 0 ? P.K : k - 1) * P.n + s) + 1;
}

// Element condensation (same elimination as elem_factor_big) with
// pair_eliminate_rt over the nt threads of the block.
// Assembly of element e's KKT block (packed lower triangle in `blk`, shared
// memory) from its derivative blocks.  Kept out of line: inlined, it changes
// how the elimination that follows is compiled (about a quarter more
// instructions there).
template <typename T>
__device__ __noinline__ void elem_assemble_rt(const DevProb& P, const DevEval& E,
                                              const double* __restrict__ sigma, double dw,
                                              double dc, int e, T* blk) {
  const int n = P.n, p = P.p, ext = P.ext, K = P.K, npt = P.np;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nn = n * n, np = n * p, ntri = ext * (ext + 1) / 2;
  const int nob = npt * npt * n, nsg = npt * n;
  // the derivative blocks arrive by asynchronous copies issued all at once
  // (one memory latency per element) while the triangle is cleared
  double* Wzz = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(blk) +
                                          elem_blk_bytes<T>(P));
  double* JZ = Wzz + K * nn;
  double* Wzt = JZ + K * nn;
  double* JT = Wzt + K * np;
  double* Wobj = JT + K * np;
  double* sig = Wobj + nob;
  {
    auto stage = [&](double* dst, const double* src, int cnt) {
      for (int i = tid; i < cnt; i += nt) cp_async_elem(dst + i, src + i);
    };
    stage(Wzz, E.Wzz + (size_t)e * K * nn, K * nn);
    stage(JZ, E.JZ + (size_t)e * K * nn, K * nn);
    stage(Wzt, E.Wzt + (size_t)e * K * np, K * np);
    stage(JT, E.JT + (size_t)e * K * np, K * np);
    stage(Wobj, E.Wobj + (size_t)e * nob, nob);
    if (sigma) stage(sig, sigma + (size_t)e * nsg, nsg);
    else
      for (int i = tid; i < nsg; i += nt) sig[i] = 0.0;
    cp_async_commit();
  }
  for (int i = tid; i < ntri; i += nt) blk[i] = T(0);
  cp_async_wait_all();
  __syncthreads();
  elem_scatter<T>(P, e, Wzz, JZ, Wzt, JT, Wobj, sig, dw, dc, blk);
}

template <typename T>
__device__ __noinline__ void elem_scatter(const DevProb& P, int e, const double* Wzz,
                                          const double* JZ, const double* Wzt, const double* JT,
                                          const double* Wobj, const double* sig, double dw,
                                          double dc, T* blk) {
  const int n = P.n, p = P.p, m = P.m, K = P.K, np = P.np;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nn = n * n, np_ = n * p;
  auto put = [&](int a, int b, T v) { blk[a >= b ? tri_at(a, b) : tri_at(b, a)] = v; };
  auto add = [&](int a, int b, T v) { blk[a >= b ? tri_at(a, b) : tri_at(b, a)] += v; };
  // 1. disjoint entries: point Hessian blocks, the identity parts of the
  //    collocation rows (D[k][j]), continuity / initial rows, -delta_c, border
  const float inv_n = 1.f / (float)n, inv_p = p > 0 ? 1.f / (float)p : 0.f;
  const float inv_np = 1.f / (float)np;
  for (int i = tid; i < K * nn; i += nt) {
    const int rs = quot(i, n, inv_n), sb = i - rs * n;   // rs = k n + sa
    const int k = quot(rs, n, inv_n), sa = rs - k * n;
    if (sa >= sb) put(loc_state(P, k + 1, sa), loc_state(P, k + 1, sb), (T)Wzz[i]);
  }
  for (int i = tid; i < K * np * n; i += nt) {
    const int kj = quot(i, n, inv_n), s2 = i - kj * n;
    const int k1 = quot(kj, np, inv_np), j = kj - k1 * np;
    put(loc_dual(P, k1 + 1, s2), loc_state(P, j, s2), (T)P.D[k1 + 1][j]);
  }
  if (!P.gauss) {
    // the element's own continuity / initial row c0 on z0
    for (int s2 = tid; s2 < n; s2 += nt) put(loc_dual(P, 0, s2), loc_state(P, 0, s2), T(1));
  } else if (chain_next(P, e)) {
    // the next element's continuity row: -b_j on every point of this element
    for (int i = tid; i < np * n; i += nt) {
      const int j = quot(i, n, inv_n), s2 = i - j * n;
      put(loc_dual(P, 0, s2), loc_state(P, j, s2), (T)(-P.bw[j]));
    }
  }
  for (int i = tid; i < np * n; i += nt) {
    const int k = quot(i, n, inv_n), s2 = i - k * n;
    const int a = loc_dual(P, k, s2);
    put(a, a, (T)(-dc));
  }
  for (int i = tid; i < K * np_; i += nt) {
    const int ks = quot(i, p, inv_p), q = i - ks * p;     // ks = k n + s
    const int k = quot(ks, n, inv_n), s2 = ks - k * n;
    put(m + q, loc_state(P, k + 1, s2), (T)Wzt[i]);
    put(m + q, loc_dual(P, k + 1, s2), (T)JT[i]);
  }
  __syncthreads();
  // 2. sums onto those: objective blocks (same species across points) and the
  //    -h df/dz part of the collocation rows
  const int np2 = np * np;
  const float inv_np2 = 1.f / (float)np2;
  for (int i = tid; i < np2 * n; i += nt) {
    const int s2 = quot(i, np2, inv_np2), jj = i - s2 * np2;
    const int ja = quot(jj, np, inv_np), jb = jj - ja * np;
    const int a = loc_state(P, ja, s2), b = loc_state(P, jb, s2);
    if (a >= b) add(a, b, (T)Wobj[i]);
  }
  for (int i = tid; i < K * nn; i += nt) {
    const int rs = quot(i, n, inv_n), sp = i - rs * n;   // rs = k n + sd
    const int k = quot(rs, n, inv_n), sd = rs - k * n;
    add(loc_dual(P, k + 1, sd), loc_state(P, k + 1, sp), (T)JZ[i]);
  }
  __syncthreads();
  // 3. barrier diagonal and delta_w on the states
  for (int i = tid; i < np * n; i += nt) {
    const int j = quot(i, n, inv_n), s2 = i - j * n;
    const int a = loc_state(P, j, s2);
    add(a, a, (T)((sig ? sig[i] : 0.0) + dw));
  }
  __syncthreads();
}

// Gauss points: the trailing chain group of element e, (z_e0, c_(e+1)0)
// pairs at local rows i0 + 2s, i0 + 2s + 1, leaves in three parts: the z part
// of chain block e (its c part and the constant identity between them are
// written here only when e starts a chain, otherwise by element e - 1), the c
// part of chain block e + 1 with the coupling Cpl[e + 1] = K[c_(e+1)0, z_e0],
// and the borders of both.  tr(a, b): the trailing block's symmetric entry.
// Out of line, so that it does not add to the register demand of the
// elimination kernels it is called from.
template <typename T, class Tr>
__device__ __noinline__ void gauss_chain_out(const DevProb& P, const DevFactor<T>& F, int e,
                                             int i0, double dc, Tr tr) {
  const int n = P.n, p = P.p, m = P.m, n2 = 2 * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool start = chain_start(P, e), next = chain_next(P, e);
  T* Ae = F.Aif + (size_t)e * n2 * n2;
  for (int i = tid; i < n * n; i += nt) {
    const int s2 = i / n, t = i - s2 * n;
    Ae[(2 * s2) * n2 + 2 * t] = tr(i0 + 2 * s2, i0 + 2 * t);
    Ae[(2 * s2) * n2 + 2 * t + 1] = s2 == t ? T(1) : T(0);
    Ae[(2 * s2 + 1) * n2 + 2 * t] = s2 == t ? T(1) : T(0);
    if (start) Ae[(2 * s2 + 1) * n2 + 2 * t + 1] = s2 == t ? (T)(-dc) : T(0);
  }
  T* Be = F.Bif + (size_t)e * n2 * p;
  for (int i = tid; i < n * p; i += nt) {
    const int s2 = i / p, q = i - s2 * p;
    Be[(2 * s2) * p + q] = tr(m + q, i0 + 2 * s2);
    if (start) Be[(2 * s2 + 1) * p + q] = T(0);
  }
  if (start) {
    T* C = F.Cpl + (size_t)e * n * n;
    for (int i = tid; i < n * n; i += nt) C[i] = T(0);
  }
  if (next) {
    T* An = F.Aif + (size_t)(e + 1) * n2 * n2;
    T* Cn = F.Cpl + (size_t)(e + 1) * n * n;
    for (int i = tid; i < n * n; i += nt) {
      const int s2 = i / n, t = i - s2 * n;
      An[(2 * s2 + 1) * n2 + 2 * t + 1] = tr(i0 + 2 * s2 + 1, i0 + 2 * t + 1);
      Cn[i] = tr(i0 + 2 * s2 + 1, i0 + 2 * t);
    }
    T* Bn = F.Bif + (size_t)(e + 1) * n2 * p;
    for (int i = tid; i < n * p; i += nt) {
      const int s2 = i / p, q = i - s2 * p;
      Bn[(2 * s2 + 1) * p + q] = tr(m + q, i0 + 2 * s2 + 1);
    }
  }
}

template <typename T, int TPT>
__device__ void elem_factor_rt(const DevProb& P, const DevEval& E,
                               const double* __restrict__ sigma, double dw, double dc,
                               const DevFactor<T>& F, int e, Pair<T>* ub, T* blk) {
  const int n = P.n, p = P.p, m = P.m, ext = P.ext;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nint = P.K * n, i0 = 2 * nint, n2 = 2 * n;
  const float inv_n = 1.f / (float)n, inv_p = p > 0 ? 1.f / (float)p : 0.f;
  elem_assemble_rt<T>(P, E, sigma, dw, dc, e, blk);
  auto entry = [&](int r, int c) -> T { return blk[tri_at(r, c)]; };
  auto sink = [&](int r, int c, T val) { blk[tri_at(r, c)] = val; };
  __shared__ Pivot<T> pivs[RT_MAX_PAIRS];
  __shared__ int cnt[3];
  pair_eliminate_rt<T, TPT, true>(tid, nt, ext, nint, entry, F.Lel + (size_t)e * (2 * nint) * ext, ext,
                            F.Del + (size_t)e * nint * 3, sink, CtaBar{}, ub, pivs, cnt);
  if (tid == 0) {
    F.inert[e * 3 + 0] = cnt[0]; F.inert[e * 3 + 1] = cnt[1]; F.inert[e * 3 + 2] = cnt[2];
  }
  // trailing block: chain block (2n x 2n, both triangles), its border (p x 2n),
  // parameter part (FP64)
  if (P.gauss) {
    __syncthreads();
    auto tr = [&](int a, int b) { return a >= b ? blk[tri_at(a, b)] : blk[tri_at(b, a)]; };
    gauss_chain_out<T>(P, F, e, i0, dc, tr);
    double* Sc = F.Scon + (size_t)e * p * p;
    for (int i = tid; i < p * p; i += nt) {
      const int q = quot(i, p, inv_p), q2 = i - q * p;
      Sc[i] = (double)(q >= q2 ? blk[tri_at(m + q, m + q2)] : blk[tri_at(m + q2, m + q)]);
    }
    return;
  }
  const float inv_n2 = 1.f / (float)n2;
  T* Aif = F.Aif + (size_t)e * n2 * n2;
  for (int i = tid; i < n2 * n2; i += nt) {
    const int u = quot(i, n2, inv_n2), v = i - u * n2;
    Aif[i] = u >= v ? blk[tri_at(i0 + u, i0 + v)] : blk[tri_at(i0 + v, i0 + u)];
  }
  T* Bif = F.Bif + (size_t)e * n2 * p;
  for (int i = tid; i < n2 * p; i += nt) {
    const int u = quot(i, p, inv_p), q = i - u * p;
    Bif[i] = blk[tri_at(m + q, i0 + u)];
  }
  double* Sc = F.Scon + (size_t)e * p * p;
  for (int i = tid; i < p * p; i += nt) {
    const int q = quot(i, p, inv_p), q2 = i - q * p;
    Sc[i] = (double)(q >= q2 ? blk[tri_at(m + q, m + q2)] : blk[tri_at(m + q2, m + q)]);
  }
  T* C = F.Cpl + (size_t)e * n * n;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int s2 = quot(idx, n, inv_n), t = idx - s2 * n;
    C[idx] = (!chain_start(P, e) && s2 == t) ? T(-1) : T(0);
  }
}

// Tile pairs per thread of elem_factor_rt (1) and its block size for an element
// of size ext (a multiple of 32 threads covering every tile; 0 when the
// element is too large and elem_factor_big is used).
template <typename T>
__host__ __device__ constexpr int rt_tpt() { return 1; }   // tile pairs per thread
template <typename T>
__host__ __device__ inline int rt_block_threads(int ext) {
  const int R = (ext + 3) >> 2;
  if (R > RT_MAX_TR) return 0;
  const int per = (tile_pairs(R) + rt_tpt<T>() - 1) / rt_tpt<T>();
  const int nt = (per + 31) / 32 * 32;
  return nt < 64 ? 64 : nt;
}

// Register cap of the element kernels: enough for the tiles, few enough for
// four (float) or two (double) blocks of 192 threads per SM.
template <typename T>
constexpr int rt_maxnreg() { return sizeof(T) == 4 ? 80 : 128; }

template <typename T>
__global__ void __maxnreg__(rt_maxnreg<T>())
k_elem_factor_rt(DevProb P, DevEval E, const double* __restrict__ sigma, double dw, double dc,
                 DevFactor<T> F) {
  __shared__ PivotBuf<T> ub;
  extern __shared__ double stage_dyn[];
  elem_factor_rt<T, rt_tpt<T>()>(P, E, sigma, dw, dc, F, blockIdx.x, ub.v,
                                 reinterpret_cast<T*>(stage_dyn));
}

// ---- 2. one level of block cyclic reduction -------------------------------------
// Eliminates the blocks at odd multiples of `stride` (final = 1: block 0 alone).
// Local order of the extended block: [interface of block i (2n) | z3 of the
// left neighbour (n) | c0 of the right neighbour (n) | theta (p)].
// Kept out of line: inside the cooperative kernel (80 registers per thread for
// the latency-bound register-tiled reduction blocks) its register demand would
// otherwise shape the whole kernel.
template <typename T, int TR, int TC>
__device__ __noinline__ void bcr_factor_big(const DevProb& P, const DevFactor<T>& F, int stride,
                                            int final_level, int bi, const BigPlace<T> pl,
                                            int pb) {
  const int n = P.n, p = P.p, N = P.N, bext = P.bext, n2 = 2 * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int i = final_level ? 0 : stride * (2 * bi + 1);
  const int L = final_level ? -1 : i - stride;
  const int R = (!final_level && i + stride < N) ? i + stride : -1;
  const T* Ai = F.Aif + (size_t)i * n2 * n2;
  const T* Ci = F.Cpl + (size_t)i * n * n;
  const T* CR = R >= 0 ? F.Cpl + (size_t)R * n * n : nullptr;
  const T* Bi = F.Bif + (size_t)i * n2 * p;
  T* A = pl.A;
  for (int a = tid >> 5; a < bext; a += nt >> 5)
    for (int b = tid & 31; b <= a; b += 32) {
      T v = T(0);
      if (a < n2) {
        v = Ai[a * n2 + b];
      } else if (b < n2) {
        if (a < 3 * n) {                       // z3 of left neighbour, t = a - 2n
          if (L >= 0 && (b & 1)) v = Ci[(b >> 1) * n + (a - n2)];
        } else if (a < 4 * n) {                // c0 of right neighbour, s = a - 3n
          if (R >= 0 && !(b & 1)) v = CR[(a - 3 * n) * n + (b >> 1)];
        } else {                               // theta row q = a - 4n
          v = Bi[b * p + (a - 4 * n)];
        }
      }
      A[tri_at(a, b)] = v;
    }
  __syncthreads();
  int pos = 0, neg = 0, zero = 0;
  pair_eliminate_big<T, TR, TC>(A, bext, n, F.Lb + (size_t)i * n2 * bext, bext,
                        F.Db + (size_t)i * n * 3, pl.Lp, pl.W, pos, neg, zero, pb);
  if (tid == 0) {
    int* in = F.inert + (size_t)(N + i) * 3;
    in[0] = pos; in[1] = neg; in[2] = zero;
  }
  // scatter the trailing (Schur) block into the neighbours
  auto tr = [&](int a, int b) { return a >= b ? A[tri_at(a, b)] : A[tri_at(b, a)]; };
  if (L >= 0) {
    T* AL = F.Aif + (size_t)L * n2 * n2;
    for (int idx = tid; idx < n * n; idx += nt) {
      const int t = idx / n, t2 = idx - t * n;
      AL[(2 * t) * n2 + 2 * t2] += tr(n2 + t, n2 + t2);
    }
    T* BL = F.Bif + (size_t)L * n2 * p;
    for (int idx = tid; idx < n * p; idx += nt) {
      const int t = idx / p, q = idx - t * p;
      BL[(2 * t) * p + q] += A[tri_at(4 * n + q, n2 + t)];
    }
  }
  if (R >= 0) {
    T* AR = F.Aif + (size_t)R * n2 * n2;
    T* CRw = F.Cpl + (size_t)R * n * n;
    for (int idx = tid; idx < n * n; idx += nt) {
      const int s2 = idx / n, s3 = idx - s2 * n;
      AR[(2 * s2 + 1) * n2 + 2 * s3 + 1] += tr(3 * n + s2, 3 * n + s3);
      CRw[idx] = (L >= 0) ? A[tri_at(3 * n + s2, n2 + s3)] : T(0);
    }
    T* BR = F.Bif + (size_t)R * n2 * p;
    for (int idx = tid; idx < n * p; idx += nt) {
      const int s2 = idx / p, q = idx - s2 * p;
      BR[(2 * s2 + 1) * p + q] += A[tri_at(4 * n + q, 3 * n + s2)];
    }
  }
  double* Sc = F.Scon + (size_t)(N + i) * p * p;
  for (int idx = tid; idx < p * p; idx += nt) {
    const int q = idx / p, q2 = idx - q * p;
    Sc[idx] = (double)tr(4 * n + q, 4 * n + q2);
  }
  __syncthreads();
}

// Cyclic-reduction block (same result as bcr_factor_big) with
// pair_eliminate_rt on one half (128 threads) of the block: tid in [0, 128).
// Its inputs are first staged in `stage` (T elements, bcr_stage_elems):
// the block's interface block [2n][2n], its coupling [n][n], the right
// neighbour's coupling [n][n] and its border [2n][p].
// After the elimination the same buffer holds the trailing block (2n + p rows,
// packed lower triangle) on its way to the neighbours.
__host__ __device__ inline size_t bcr_stage_elems(int n, int p) {
  const size_t in = 6 * (size_t)n * n + 2 * (size_t)n * p, m2 = 2 * (size_t)n + p;
  const size_t out = m2 * (m2 + 1) / 2;
  return in > out ? in : out;
}
// Starts the staging of cyclic-reduction block bi's inputs into `stage` (one
// half, tid in [0, 128)); the copies are complete for this thread after
// cp_async_wait_all and for the half after a barrier that follows it.  A
// block's inputs are not written by any other block of its level, so they
// can be staged while the half still works on its previous block.
template <typename T>
__device__ void bcr_stage_issue(const DevProb& P, const DevFactor<T>& F, int stride,
                                int final_level, int bi, int tid, T* stage) {
  const int n = P.n, p = P.p, N = P.N, n2 = 2 * n;
  const int i = final_level ? 0 : stride * (2 * bi + 1);
  const int R = (!final_level && i + stride < N) ? i + stride : -1;
  T* Ai = stage;
  T* Ci = Ai + 4 * n * n;
  T* CR = Ci + n * n;
  T* Bi = CR + n * n;
  const T* gA = F.Aif + (size_t)i * n2 * n2;
  const T* gC = F.Cpl + (size_t)i * n * n;
  const T* gCR = R >= 0 ? F.Cpl + (size_t)R * n * n : nullptr;
  const T* gB = F.Bif + (size_t)i * n2 * p;
  for (int k = tid; k < 4 * n * n; k += 128) cp_async_elem(Ai + k, gA + k);
  for (int k = tid; k < n * n; k += 128) {
    cp_async_elem(Ci + k, gC + k);
    if (gCR) cp_async_elem(CR + k, gCR + k);
    else CR[k] = T(0);
  }
  for (int k = tid; k < n2 * p; k += 128) cp_async_elem(Bi + k, gB + k);
  cp_async_commit();
}

// Factorization of a block whose inputs are staged (complete and visible to
// the half).
template <typename T, int TPT>
__device__ void bcr_factor_staged(const DevProb& P, const DevFactor<T>& F, int stride,
                                  int final_level, int bi, int tid, HalfBar bar, Pair<T>* ub,
                                  T* stage, Pivot<T>* pivs, int* cnt) {
  const int n = P.n, p = P.p, N = P.N, bext = P.bext, n2 = 2 * n;
  const int i = final_level ? 0 : stride * (2 * bi + 1);
  const int L = final_level ? -1 : i - stride;
  const int R = (!final_level && i + stride < N) ? i + stride : -1;
  T* Ai = stage;
  T* Ci = Ai + 4 * n * n;
  T* CR = Ci + n * n;
  T* Bi = CR + n * n;
  auto entry = [&](int a, int b) -> T {
    if (a < n2) return Ai[a * n2 + b];
    if (b >= n2) return T(0);
    if (a < 3 * n)                 // z3 of left neighbour, t = a - 2n
      return (L >= 0 && (b & 1)) ? Ci[(b >> 1) * n + (a - n2)] : T(0);
    if (a < 4 * n)                 // c0 of right neighbour, s = a - 3n
      return (R >= 0 && !(b & 1)) ? CR[(a - 3 * n) * n + (b >> 1)] : T(0);
    return Bi[b * p + (a - 4 * n)];  // theta row q = a - 4n
  };
  // the trailing (Schur) block, local rows [z3 of L (n) | c0 of R (n) | theta (p)],
  // is collected in the staging buffer (the inputs are in registers by now) ...
  const int b2 = 2 * n;
  auto sink = [&](int r, int c, T val) { stage[tri_at(r - b2, c - b2)] = val; };
  pair_eliminate_rt<T, TPT, false>(tid, 128, bext, n, entry, F.Lb + (size_t)i * n2 * bext, bext,
                            F.Db + (size_t)i * n * 3, sink, bar, ub, pivs, cnt);
  if (tid == 0) {
    int* in = F.inert + (size_t)(N + i) * 3;
    in[0] = cnt[0]; in[1] = cnt[1]; in[2] = cnt[2];
  }
  // ... and added into the neighbours in coalesced passes of independent
  // read-modify-writes: z3 x z3 into the left neighbour's interface block and
  // border, c0 x c0 into the right one's, the new coupling c0(R) x z3(L), and
  // the p x p part into this block's parameter contribution
  auto tr = [&](int a, int b) { return a >= b ? stage[tri_at(a, b)] : stage[tri_at(b, a)]; };
  const float inv_n = 1.f / (float)n, inv_p = p > 0 ? 1.f / (float)p : 0.f;
  if (L >= 0) {
    T* AL = F.Aif + (size_t)L * n2 * n2;
    for (int k = tid; k < n * n; k += 128) {
      const int t = quot(k, n, inv_n), t2 = k - t * n;
      AL[(2 * t) * n2 + 2 * t2] += tr(t, t2);
    }
    T* BL = F.Bif + (size_t)L * n2 * p;
    for (int k = tid; k < n * p; k += 128) {
      const int t = quot(k, p, inv_p), q = k - t * p;
      BL[(2 * t) * p + q] += tr(2 * n + q, t);
    }
  }
  if (R >= 0) {
    T* AR = F.Aif + (size_t)R * n2 * n2;
    T* CRw = F.Cpl + (size_t)R * n * n;
    for (int k = tid; k < n * n; k += 128) {
      const int s2 = quot(k, n, inv_n), t = k - s2 * n;
      AR[(2 * s2 + 1) * n2 + 2 * t + 1] += tr(n + s2, n + t);
      CRw[k] = L >= 0 ? tr(n + s2, t) : T(0);
    }
    T* BR = F.Bif + (size_t)R * n2 * p;
    for (int k = tid; k < n * p; k += 128) {
      const int s2 = quot(k, p, inv_p), q = k - s2 * p;
      BR[(2 * s2 + 1) * p + q] += tr(2 * n + q, n + s2);
    }
  }
  double* Sc = F.Scon + (size_t)(N + i) * p * p;
  for (int k = tid; k < p * p; k += 128) {
    const int q = quot(k, p, inv_p), q2 = k - q * p;
    Sc[k] = (double)tr(2 * n + q, 2 * n + q2);
  }
  bar();   // the buffer is restaged by this half's next block
}

// bcr_factor_staged with its staging waited for (no overlap).
template <typename T, int TPT>
__device__ void bcr_factor_rt(const DevProb& P, const DevFactor<T>& F, int stride,
                              int final_level, int bi, int tid, HalfBar bar, Pair<T>* ub,
                              T* stage, Pivot<T>* pivs, int* cnt) {
  bcr_stage_issue<T>(P, F, stride, final_level, bi, tid, stage);
  cp_async_wait_all();
  bar();
  bcr_factor_staged<T, TPT>(P, F, stride, final_level, bi, tid, bar, ub, stage, pivs, cnt);
}

// Tiles per thread of bcr_factor_rt for P (single tiles; 0: use bcr_factor_big).
__host__ __device__ inline int bcr_rt_tiles(int bext) {
  const int R = (bext + 3) >> 2;
  if (R > RT_MAX_TR) return 0;
  const int tpt = (R * (R + 1) / 2 + 127) / 128;
  return tpt <= 2 ? tpt : 0;
}

__host__ __device__ inline int bcr_level_blocks(int N, int stride) {
  return (N - stride + 2 * stride - 1) / (2 * stride);
}

template <typename T, int BT>
__global__ void __launch_bounds__(FBS)
k_bcr_factor(DevProb P, DevFactor<T> F, int stride, int final_level, int use_smem, int slab_pb) {
  extern __shared__ unsigned char smraw[];
  const int nblk = final_level ? 1 : bcr_level_blocks(P.N, stride);
  if constexpr (BT > 0) {
    // two blocks of the level per CUDA block, one per half
    __shared__ PivotBuf<T> ub[2];
    __shared__ Pivot<T> pivs[2][RT_MAX_PAIRS];
    __shared__ int cnt[2][3];
    const int half = threadIdx.x >> 7;
    T* stage = reinterpret_cast<T*>(smraw) + half * bcr_stage_elems(P.n, P.p);
    for (int bi = 2 * blockIdx.x + half; bi < nblk; bi += 2 * gridDim.x)
      bcr_factor_rt<T, BT>(P, F, stride, final_level, bi, threadIdx.x & 127, HalfBar{1 + half},
                           ub[half].v, stage, pivs[half], cnt[half]);
  } else {
    const BigPlace<T> pl = big_place<T>(smraw, F.work, P.bext, use_smem != 0);
    for (int bi = blockIdx.x; bi < nblk; bi += gridDim.x)
      bcr_factor_big<T, 8, sizeof(T) == 4 ? 8 : 4>(P, F, stride, final_level, bi, pl,
                                                    use_smem ? 8 : slab_pb);
  }
}

// ---- 3. parameter Schur complement (FP64) ------------------------------------------
// part[g][l] = sum of X[c][l] over the g-th of G contiguous chunks of c.
constexpr int CS_BS = 256;
__device__ inline double chunk_sum_item(const double* __restrict__ X, int C, int L, int G, int g,
                                        int l) {
  const int c0 = (int)((long long)C * g / G), c1 = (int)((long long)C * (g + 1) / G);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int c = c0;
  for (; c + 3 < c1; c += 4) {
    a0 += X[(size_t)c * L + l];
    a1 += X[(size_t)(c + 1) * L + l];
    a2 += X[(size_t)(c + 2) * L + l];
    a3 += X[(size_t)(c + 3) * L + l];
  }
  for (; c < c1; ++c) a0 += X[(size_t)c * L + l];
  return (a0 + a1) + (a2 + a3);
}

__global__ void __launch_bounds__(CS_BS)
k_chunk_sums(const double* __restrict__ X, int C, int L, int G, double* __restrict__ part) {
  const int l = blockIdx.x * CS_BS + threadIdx.x;
  const int g = blockIdx.y;
  if (l >= L) return;
  part[(size_t)g * L + l] = chunk_sum_item(X, C, L, G, g, l);
}

cudaError_t launch_chunk_sums(const double* X, int C, int L, double* part, cudaStream_t st) {
  if (L <= 0) return cudaSuccess;
  dim3 grid(ceil_div(L, CS_BS), n_chunks(C));
  count_launch();
  k_chunk_sums<<<grid, CS_BS, 0, st>>>(X, C, L, n_chunks(C), part);
  return cudaGetLastError();
}

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

constexpr int SBS = 256;
// One block: S = (chunk sums of all contributions) + diag(W_thth + sigma + dw),
// FP64 LDL^T with 1x1 pivots, total inertia.  sS: [p][p] followed by a
// p-entry multiplier row, in dynamic shared memory, or S.S itself when that
// does not fit (S.S holds p p + p doubles for this).
__device__ void schur_block(const DevProb& P, const int* __restrict__ inert,
                            const double* __restrict__ chunkS, const double* __restrict__ wtt,
                            const double* __restrict__ sigma, double dw, const DevSchur& S,
                            double* sS) {
  __shared__ long long cnt[3];
  __shared__ long long red[3][SBS];
  const int p = P.p, N = P.N, tid = threadIdx.x;
  const size_t nz = (size_t)N * P.np * P.n;
  double* l = sS + (size_t)p * p;
  for (int idx = tid; idx < p * p; idx += SBS) {
    const int q = idx / p, q2 = idx - q * p;
    double v = sum_chunks(chunkS, n_chunks(2 * N), p * p, idx);
    if (q == q2) v += wtt[q] + (sigma ? sigma[nz + q] : 0.0) + dw;
    sS[idx] = v;
  }
  {
    long long a = 0, b = 0, c = 0;
    for (int k = tid; k < 2 * N; k += SBS) { a += inert[3 * k]; b += inert[3 * k + 1]; c += inert[3 * k + 2]; }
    red[0][tid] = a; red[1][tid] = b; red[2][tid] = c;
    __syncthreads();
    for (int s = SBS / 2; s > 0; s >>= 1) {
      if (tid < s) { red[0][tid] += red[0][tid + s]; red[1][tid] += red[1][tid + s]; red[2][tid] += red[2][tid + s]; }
      __syncthreads();
    }
    if (tid == 0) { cnt[0] = red[0][0]; cnt[1] = red[1][0]; cnt[2] = red[2][0]; }
  }
  __syncthreads();
  for (int k = 0; k < p; ++k) {
    const double d = sS[k * p + k];
    const bool ok = (d != 0.0) && isfinite(d);
    const double inv = ok ? 1.0 / d : 0.0;
    for (int r = k + 1 + tid; r < p; r += SBS) l[r] = sS[r * p + k] * inv;
    if (tid == 0) {
      if (!ok) cnt[2] += 1; else if (d > 0) cnt[0] += 1; else cnt[1] += 1;
      S.Sd[k] = d;
    }
    __syncthreads();
    const int w = p - k - 1;
    for (int idx = tid; idx < w * w; idx += SBS) {
      const int r = k + 1 + idx / w, c = k + 1 + idx % w;
      if (c <= r) sS[r * p + c] -= l[r] * sS[c * p + k];
    }
    __syncthreads();
    for (int r = k + 1 + tid; r < p; r += SBS) sS[r * p + k] = l[r];
    __syncthreads();
  }
  for (int idx = tid; idx < p * p; idx += SBS) S.S[idx] = sS[idx];
  if (tid == 0) { S.inertia[0] = cnt[0]; S.inertia[1] = cnt[1]; S.inertia[2] = cnt[2]; }
  __syncthreads();
}

__global__ void __launch_bounds__(SBS)
k_schur(DevProb P, const int* __restrict__ inert, const double* __restrict__ chunkS,
        const double* __restrict__ wtt, const double* __restrict__ sigma, double dw,
        DevSchur S, int in_global) {
  extern __shared__ double sS[];
  schur_block(P, inert, chunkS, wtt, sigma, dw, S, in_global ? S.S : sS);
}

// ---- solves: one warp per block ----------------------------------------------------
constexpr int SOLVE_WARPS = 4;

template <typename T>
__device__ inline void pair_solve_d(T a, T b, T d, T w0, T w1, T& v0, T& v1) {
  const T det = fma(a, d, -(b * b));
  if (det != T(0) && isfinite(det)) {
    const T inv = recip_rn(det);
    v0 = fma(d, w0, -(b * w1)) * inv;
    v1 = fma(a, w1, -(b * w0)) * inv;
  } else {
    v0 = T(0); v1 = T(0);
  }
}

// Substitutions through a block's eliminated pairs, one warp per block.  The
// work is a sequence of items: pair q (columns 2q, 2q+1 of L, stored as
// Lc[c * lds + r]) restricted to one chunk of SUB_J * 32 of its rows below the
// pair.  The L values of an item do not depend on the vector being solved, so
// they are loaded SUB_D items ahead into a register ring: each warp keeps
// several loads in flight instead of waiting a memory latency per pair.  Per
// row, the arithmetic and its order are those of the plain column loop.
constexpr int SUB_J = 4;   // rows per lane in one item (chunks of 128 rows)
constexpr int SUB_D = 2;   // items loaded ahead

__device__ inline int sub_chunks(int msz, int q) {
  const int rows = msz - 2 * q - 2;
  return rows > 0 ? (rows + 32 * SUB_J - 1) / (32 * SUB_J) : 0;
}

template <typename T>
__device__ inline void sub_fetch(const T* __restrict__ Lc, int lds, int msz, int q, int k, bool ok,
                                 T (&a)[SUB_J], T (&b)[SUB_J]) {
  const int lane = threadIdx.x & 31;
  const T* L0 = Lc + (size_t)(2 * q) * lds;
  const T* L1 = L0 + lds;
  const int r0 = 2 * q + 2 + 32 * SUB_J * k + lane;
#pragma unroll
  for (int j = 0; j < SUB_J; ++j) {
    const int r = r0 + 32 * j;
    const bool in = ok && r < msz;
    a[j] = in ? L0[r] : T(0);
    b[j] = in ? L1[r] : T(0);
  }
}

// Forward substitution: w (length msz) in shared memory; after the call w
// holds L^{-1} w.  Items run over pairs ascending, chunks ascending.
template <typename T>
__device__ void warp_forward(T* w, int msz, int npairs, const T* __restrict__ Lc, int lds) {
  const int lane = threadIdx.x & 31;
  // consumer and prefetch cursors (pair, chunk); a pair without rows below
  // it ends the sequence, since every later pair has fewer rows
  int cq = 0, ck = 0, fq = 0, fk = 0;
  auto valid = [&](int q) { return q < npairs && sub_chunks(msz, q) > 0; };
  auto advance = [&](int& q, int& k) {
    if (++k >= sub_chunks(msz, q)) { ++q; k = 0; }
  };
  T a[SUB_D][SUB_J], b[SUB_D][SUB_J];
#pragma unroll
  for (int s = 0; s < SUB_D; ++s) {
    const bool ok = valid(fq);
    sub_fetch<T>(Lc, lds, msz, fq, fk, ok, a[s], b[s]);
    if (ok) advance(fq, fk);
  }
  while (valid(cq)) {
#pragma unroll
    for (int s = 0; s < SUB_D; ++s) {
      if (valid(cq)) {
        __syncwarp();
        const T w0 = w[2 * cq], w1 = w[2 * cq + 1];
        const int r0 = 2 * cq + 2 + 32 * SUB_J * ck + lane;
#pragma unroll
        for (int j = 0; j < SUB_J; ++j) {
          const int r = r0 + 32 * j;
          if (r < msz) w[r] = fma(-b[s][j], w1, fma(-a[s][j], w0, w[r]));
        }
        const bool ok = valid(fq);
        sub_fetch<T>(Lc, lds, msz, fq, fk, ok, a[s], b[s]);
        if (ok) advance(fq, fk);
        advance(cq, ck);
      }
    }
  }
  __syncwarp();
}

// Back substitution: x (length msz) holds the known tail values; pairs are
// solved from the last to the first: x_q = v_q - sum_{r > q} L[r][q] x_r.
// Every pair is at least one item, so that pairs without rows below them
// are solved too.
template <typename T>
__device__ void warp_backward(T* x, const T* v, int msz, int npairs, const T* __restrict__ Lc,
                              int lds) {
  const int lane = threadIdx.x & 31;
  auto nitems = [&](int q) { return max(1, sub_chunks(msz, q)); };
  int cq = npairs - 1, ck = 0, fq = npairs - 1, fk = 0;
  auto advance = [&](int& q, int& k) {
    if (++k >= nitems(q)) { --q; k = 0; }
  };
  T a[SUB_D][SUB_J], b[SUB_D][SUB_J];
#pragma unroll
  for (int s = 0; s < SUB_D; ++s) {
    const bool ok = fq >= 0;
    sub_fetch<T>(Lc, lds, msz, ok ? fq : 0, fk, ok, a[s], b[s]);
    if (ok) advance(fq, fk);
  }
  T s0 = T(0), s1 = T(0);
  while (cq >= 0) {
#pragma unroll
    for (int s = 0; s < SUB_D; ++s) {
      if (cq >= 0) {
        const int r0 = 2 * cq + 2 + 32 * SUB_J * ck + lane;
#pragma unroll
        for (int j = 0; j < SUB_J; ++j) {
          const int r = r0 + 32 * j;
          if (r < msz) {
            const T xr = x[r];
            s0 = fma(a[s][j], xr, s0);
            s1 = fma(b[s][j], xr, s1);
          }
        }
        const bool ok = fq >= 0;
        sub_fetch<T>(Lc, lds, msz, ok ? fq : 0, fk, ok, a[s], b[s]);
        if (ok) advance(fq, fk);
        if (ck + 1 >= nitems(cq)) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
          }
          if (lane == 0) { x[2 * cq] = v[2 * cq] - s0; x[2 * cq + 1] = v[2 * cq + 1] - s1; }
          s0 = T(0); s1 = T(0);
          __syncwarp();
        }
        advance(cq, ck);
      }
    }
  }
}

// local index a < m -> position in the API-layout KKT vector of element e.
// Radau: every local row is an unknown of the element.
__device__ inline size_t elem_global(const DevProb& P, int e, int a) {
  const int n = P.n;
  const size_t nx = (size_t)P.N * 4 * n + P.p;
  const int pr = a >> 1, g = pr / n, s = pr - g * n;
  if (a & 1) return nx + ((size_t)e * 4 + grp_con(0, 3, g)) * n + s;
  return ((size_t)e * 4 + grp_point(0, 3, g)) * n + s;
}
// Gauss: the chain group's multipliers are the next element's c0, absent
// (-1) after a chain's last element, whose block has zero rows there apart
// from -delta_c.
__device__ inline long long elem_global_gauss(const DevProb& P, int e, int a) {
  const int n = P.n, np = P.np;
  const size_t nx = (size_t)P.N * np * n + P.p;
  const int pr = a >> 1, g = pr / n, s = pr - g * n;
  if (a & 1) {
    if (g == P.K) return chain_next(P, e) ? (long long)(nx + (size_t)(e + 1) * np * n + s) : -1;
    return (long long)(nx + ((size_t)e * np + g + 1) * n + s);
  }
  return (long long)(((size_t)e * np + (g < P.K ? g + 1 : 0)) * n + s);
}
// w[a] = v[global index of a] (0 where there is none) for a in [lo, hi), or
// the reverse when store (Gauss elements, one warp; out of line).
template <typename T>
__device__ __noinline__ void gauss_elem_gather(const DevProb& P, int e, const double* v, T* w,
                                               int lo, int hi) {
  for (int a = lo + (threadIdx.x & 31); a < hi; a += 32) {
    const long long gi = elem_global_gauss(P, e, a);
    w[a] = gi >= 0 ? (T)v[gi] : T(0);
  }
}
template <typename T>
__device__ __noinline__ void gauss_elem_scatter(const DevProb& P, int e, const T* w, double* v,
                                                int lo, int hi) {
  for (int a = lo + (threadIdx.x & 31); a < hi; a += 32) {
    const long long gi = elem_global_gauss(P, e, a);
    if (gi >= 0) v[gi] = (double)w[a];
  }
}

// Gauss points: chain right-hand sides after element e's forward
// elimination (wt: the trailing rows (z_e0, c_(e+1)0) interleaved): the z part
// of chain block e and the c part of chain block e + 1 (the rhs of c_(e+1)0
// updated by this element's elimination); a chain's first element also sets
// its own c part, the rhs of its initial condition.  One warp.
template <typename T>
__device__ __noinline__ void gauss_chain_rhs(const DevProb& P, const DevFactor<T>& F,
                                             const double* __restrict__ b, int e, const T* wt) {
  const int lane = threadIdx.x & 31, n = P.n;
  const size_t nx = (size_t)P.N * P.np * n + P.p;
  T* Rif = F.Rif + (size_t)e * 2 * n;
  const bool start = chain_start(P, e), next = chain_next(P, e);
  for (int s2 = lane; s2 < n; s2 += 32) {
    Rif[2 * s2] = wt[2 * s2];
    if (start) Rif[2 * s2 + 1] = (T)b[nx + (size_t)e * P.np * n + s2];
    if (next) F.Rif[(size_t)(e + 1) * 2 * n + 2 * s2 + 1] = wt[2 * s2 + 1];
  }
}

template <typename T>
__device__ void elem_fwd_one(const DevProb& P, const DevFactor<T>& F, const double* __restrict__ b,
                             int e, T* w) {
  const int lane = threadIdx.x & 31;
  const int n = P.n, ext = P.ext, m = P.m, p = P.p;
  if (!P.gauss) {
    for (int a = lane; a < ext; a += 32) w[a] = a < m ? (T)b[elem_global(P, e, a)] : T(0);
  } else {
    gauss_elem_gather<T>(P, e, b, w, 0, m);
    for (int a = m + lane; a < ext; a += 32) w[a] = T(0);
  }
  __syncwarp();
  const int nint = P.K * n;
  const T* Lc = F.Lel + (size_t)e * (2 * nint) * ext;
  warp_forward<T>(w, ext, nint, Lc, ext);
  const T* D = F.Del + (size_t)e * nint * 3;
  T* V = F.Vint + (size_t)e * 2 * nint;
  for (int q = lane; q < nint; q += 32) {
    T v0, v1;
    pair_solve_d<T>(D[3 * q], D[3 * q + 1], D[3 * q + 2], w[2 * q], w[2 * q + 1], v0, v1);
    V[2 * q] = v0; V[2 * q + 1] = v1;
  }
  T* Rif = F.Rif + (size_t)e * 2 * n;
  if (!P.gauss) {
    for (int u = lane; u < 2 * n; u += 32) Rif[u] = w[2 * nint + u];
  } else {
    gauss_chain_rhs<T>(P, F, b, e, w + 2 * nint);
  }
  double* Rth = F.Rth + (size_t)e * p;
  for (int q = lane; q < p; q += 32) Rth[q] = (double)w[m + q];
  __syncwarp();
}

template <typename T>
__device__ void bcr_fwd_one(const DevProb& P, const DevFactor<T>& F, int stride, int final_level,
                            int bi, T* w) {
  const int lane = threadIdx.x & 31;
  const int n = P.n, p = P.p, N = P.N, bext = P.bext, n2 = 2 * n;
  const int i = final_level ? 0 : stride * (2 * bi + 1);
  const int L = final_level ? -1 : i - stride;
  const int R = (!final_level && i + stride < N) ? i + stride : -1;
  const T* Rii = F.Rif + (size_t)i * n2;
  for (int a = lane; a < bext; a += 32) w[a] = a < n2 ? Rii[a] : T(0);
  __syncwarp();
  warp_forward<T>(w, bext, n, F.Lb + (size_t)i * n2 * bext, bext);
  const T* D = F.Db + (size_t)i * n * 3;
  T* V = F.Vb + (size_t)i * n2;
  for (int q = lane; q < n; q += 32) {
    T v0, v1;
    pair_solve_d<T>(D[3 * q], D[3 * q + 1], D[3 * q + 2], w[2 * q], w[2 * q + 1], v0, v1);
    V[2 * q] = v0; V[2 * q + 1] = v1;
  }
  if (L >= 0) {
    T* RL = F.Rif + (size_t)L * n2;
    for (int t = lane; t < n; t += 32) RL[2 * t] += w[n2 + t];
  }
  if (R >= 0) {
    T* RR = F.Rif + (size_t)R * n2;
    for (int s = lane; s < n; s += 32) RR[2 * s + 1] += w[3 * n + s];
  }
  double* Rth = F.Rth + (size_t)(N + i) * p;
  for (int q = lane; q < p; q += 32) Rth[q] = (double)w[4 * n + q];
  __syncwarp();
}

// Parameter solve by one block: rhs = b_theta + chunk sums of the
// contributions, then the FP64 LDL^T of the Schur complement (column-oriented
// substitutions, one barrier per column).  sv: dynamic shared [p].
__device__ void theta_solve_block(const DevProb& P, const double* __restrict__ chunkR,
                                  const double* __restrict__ b, const DevSchur& S,
                                  double* __restrict__ sol, double* sv) {
  const int p = P.p, N = P.N, tid = threadIdx.x;
  const size_t nz = (size_t)N * P.np * P.n;
  for (int q = tid; q < p; q += blockDim.x) sv[q] = b[nz + q] + sum_chunks(chunkR, n_chunks(2 * N), p, q);
  __syncthreads();
  for (int k = 0; k < p; ++k) {
    const double xk = sv[k];
    for (int r = k + 1 + tid; r < p; r += blockDim.x) sv[r] -= S.S[r * p + k] * xk;
    __syncthreads();
  }
  for (int k = tid; k < p; k += blockDim.x) {
    const double d = S.Sd[k];
    sv[k] = (d != 0.0 && isfinite(d)) ? sv[k] / d : 0.0;
  }
  __syncthreads();
  for (int k = p - 1; k >= 0; --k) {
    const double xk = sv[k];
    for (int r = tid; r < k; r += blockDim.x) sv[r] -= S.S[k * p + r] * xk;
    __syncthreads();
  }
  for (int q = tid; q < p; q += blockDim.x) { sol[nz + q] = sv[q]; S.xth[q] = sv[q]; }
  __syncthreads();
}

__global__ void __launch_bounds__(SBS)
k_theta_solve(DevProb P, const double* __restrict__ chunkR, const double* __restrict__ b,
              DevSchur S, double* __restrict__ sol) {
  extern __shared__ double sv[];
  theta_solve_block(P, chunkR, b, S, sol, sv);
}

template <typename T>
__device__ void bcr_bwd_one(const DevProb& P, const DevFactor<T>& F, const DevSchur& S,
                            double* __restrict__ sol, int stride, int final_level, int bi, T* x) {
  const int lane = threadIdx.x & 31;
  const int n = P.n, p = P.p, N = P.N, bext = P.bext, n2 = 2 * n, np = P.np, cpt = P.cpt;
  const int i = final_level ? 0 : stride * (2 * bi + 1);
  const int L = final_level ? -1 : i - stride;
  const int R = (!final_level && i + stride < N) ? i + stride : -1;
  const size_t nx = (size_t)N * np * n + p;
  for (int a = lane; a < bext; a += 32) {
    T v = T(0);
    if (a >= n2 && a < 3 * n) {
      if (L >= 0) v = (T)sol[((size_t)L * np + cpt) * n + (a - n2)];
    } else if (a >= 3 * n && a < 4 * n) {
      if (R >= 0) v = (T)sol[nx + (size_t)R * np * n + (a - 3 * n)];
    } else if (a >= 4 * n) {
      v = (T)S.xth[a - 4 * n];
    }
    x[a] = v;
  }
  __syncwarp();
  warp_backward<T>(x, F.Vb + (size_t)i * n2, bext, n, F.Lb + (size_t)i * n2 * bext, bext);
  for (int s = lane; s < n; s += 32) {
    sol[((size_t)i * np + cpt) * n + s] = (double)x[2 * s];
    sol[nx + (size_t)i * np * n + s] = (double)x[2 * s + 1];
  }
  __syncwarp();
}

template <typename T>
__device__ void elem_bwd_one(const DevProb& P, const DevFactor<T>& F, const DevSchur& S,
                             double* __restrict__ sol, int e, T* x) {
  const int lane = threadIdx.x & 31;
  const int n = P.n, ext = P.ext, m = P.m;
  const int nint = P.K * n;
  if (!P.gauss) {
    for (int a = lane; a < ext; a += 32) {
      T v = T(0);
      if (a >= 2 * nint && a < m) v = (T)sol[elem_global(P, e, a)];
      else if (a >= m) v = (T)S.xth[a - m];
      x[a] = v;
    }
  } else {
    for (int a = lane; a < 2 * nint; a += 32) x[a] = T(0);
    gauss_elem_gather<T>(P, e, sol, x, 2 * nint, m);
    for (int a = m + lane; a < ext; a += 32) x[a] = (T)S.xth[a - m];
  }
  __syncwarp();
  warp_backward<T>(x, F.Vint + (size_t)e * 2 * nint, ext, nint,
                   F.Lel + (size_t)e * (2 * nint) * ext, ext);
  if (!P.gauss)
    for (int a = lane; a < 2 * nint; a += 32) sol[elem_global(P, e, a)] = (double)x[a];
  else
    gauss_elem_scatter<T>(P, e, x, sol, 0, 2 * nint);
  __syncwarp();
}

template <typename T>
__global__ void __launch_bounds__(32 * SOLVE_WARPS)
k_elem_fwd(DevProb P, DevFactor<T> F, const double* __restrict__ b) {
  extern __shared__ unsigned char smraw[];
  const int warp = threadIdx.x >> 5;
  const int e = blockIdx.x * SOLVE_WARPS + warp;
  if (e >= P.N) return;
  elem_fwd_one<T>(P, F, b, e, reinterpret_cast<T*>(smraw) + (size_t)warp * P.ext);
}

template <typename T>
__global__ void __launch_bounds__(32 * SOLVE_WARPS)
k_bcr_fwd(DevProb P, DevFactor<T> F, int stride, int final_level) {
  extern __shared__ unsigned char smraw[];
  const int warp = threadIdx.x >> 5;
  const int nblk = final_level ? 1 : bcr_level_blocks(P.N, stride);
  const int bi = blockIdx.x * SOLVE_WARPS + warp;
  if (bi >= nblk) return;
  bcr_fwd_one<T>(P, F, stride, final_level, bi, reinterpret_cast<T*>(smraw) + (size_t)warp * P.bext);
}

template <typename T>
__global__ void __launch_bounds__(32 * SOLVE_WARPS)
k_bcr_bwd(DevProb P, DevFactor<T> F, DevSchur S, double* __restrict__ sol, int stride,
          int final_level) {
  extern __shared__ unsigned char smraw[];
  const int warp = threadIdx.x >> 5;
  const int nblk = final_level ? 1 : bcr_level_blocks(P.N, stride);
  const int bi = blockIdx.x * SOLVE_WARPS + warp;
  if (bi >= nblk) return;
  bcr_bwd_one<T>(P, F, S, sol, stride, final_level, bi,
                 reinterpret_cast<T*>(smraw) + (size_t)warp * P.bext);
}

template <typename T>
__global__ void __launch_bounds__(32 * SOLVE_WARPS)
k_elem_bwd(DevProb P, DevFactor<T> F, DevSchur S, double* __restrict__ sol) {
  extern __shared__ unsigned char smraw[];
  const int warp = threadIdx.x >> 5;
  const int e = blockIdx.x * SOLVE_WARPS + warp;
  if (e >= P.N) return;
  elem_bwd_one<T>(P, F, S, sol, e, reinterpret_cast<T*>(smraw) + (size_t)warp * P.ext);
}

// ---- persistent cooperative kernels ------------------------------------------------
// A whole factorization or a whole solve in one cooperative launch: the phases
// of the elimination tree (elements, each cyclic-reduction level, the
// parameter block) are separated by a grid barrier instead of kernel
// boundaries.  Barrier e of a launch completes when the arrival counter
// reaches (e + 1) * gridDim.x: a block arrives with one release reduction
// and waits by polling the counter (no returning atomic on the way, nothing
// to reset between barriers).  The last block to leave the kernel zeroes the
// counter for the next launch.  The wait is bounded: after GridBar::spin_limit
// polls (GRID_SPIN_LIMIT when 0) it records an error in GridBar::err and
// continues, so a fault shows up as a status on the host instead of a hang.
constexpr long long GRID_SPIN_LIMIT = 20000000;   // ~1-2 s of polling

__device__ inline unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// `epoch` counts the barriers this block has passed in the launch.
__device__ void grid_barrier(GridBar* gb, unsigned int& epoch) {
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    // extra and spin_limit are set by the host before the launch
    const unsigned int target = epoch * gridDim.x + gb->extra;
    const long long limit = gb->spin_limit > 0 ? gb->spin_limit : GRID_SPIN_LIMIT;
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&gb->count) : "memory");
    long long spins = 0;
    while (ld_acquire_gpu(&gb->count) < target) {
      __nanosleep(32);
      if (++spins > limit) { atomicExch(&gb->err, 1); break; }
    }
  }
  __syncthreads();
}

// Called by every block as its last statement: every block has passed every
// barrier once the exit count reaches gridDim.x, so the counters can be zeroed.
__device__ void grid_exit(GridBar* gb) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int left = atomicAdd(&gb->exits, 1u) + 1u;
    if (left == gridDim.x) {
      atomicExch(&gb->count, 0u);
      atomicExch(&gb->exits, 0u);
    }
  }
}

// ---- batched persistent kernels -------------------------------------------------------
// Work of all active instances of a batch in one cooperative launch.  Plan
// arrays (device memory, written by the host):
//   pre_elem[A+1]       prefix of element counts
//   pre_lv[l][A+1]      prefix of cyclic-reduction blocks eliminated at level l
//   pre_cs[A+1]         prefix of chunk-sum items (chunks x p^2 for the factor,
//                       chunks x p for the solve)
// Per-instance flags (InstFlags) say whether that instance's blocks fit the
// kernel's shared memory or use its global slabs.
template <typename T>
__device__ inline const DevFactor<T>& inst_factor(const DevInst& I);
template <>
__device__ inline const DevFactor<float>& inst_factor<float>(const DevInst& I) { return I.F32; }
template <>
__device__ inline const DevFactor<double>& inst_factor<double>(const DevInst& I) { return I.F64; }

// Element condensation of a batch with elem_factor_rt: one block per element of
// the work list; instances without flag 4 are condensed inside k_factor_b.
template <typename T>
__global__ void __maxnreg__(rt_maxnreg<T>())
k_elem_factor_rt_b(const DevInst* __restrict__ insts, const int* __restrict__ act, int A,
                   const int* __restrict__ pre_elem, const InstParams* __restrict__ prm,
                   const int* __restrict__ flags) {
  __shared__ PivotBuf<T> ub;
  extern __shared__ double stage_dyn[];
  const int t = blockIdx.x;
  const int k = find_item(pre_elem, A, t);
  if (!(flags[k] & 4)) return;
  const DevInst& I = insts[act[k]];
  elem_factor_rt<T, rt_tpt<T>()>(I.P, I.E, I.sigma, prm[k].dw, prm[k].dc, inst_factor<T>(I),
                                 t - pre_elem[k], ub.v, reinterpret_cast<T*>(stage_dyn));
}

// Element condensation of a batch for the instances whose element blocks are
// above the register-tile limit (without flag 4): elements of the work list
// taken in turn by the CUDA blocks of the grid (at most one global slab per
// CUDA block), block storage in shared memory (flag 1) or in the slab.
// BS threads per block (Schedule::big_threads): 512 with one block per SM, or
// 256 compiled for two blocks per SM (128 registers per thread), so that where
// the shared memory allows, two elements are condensed on an SM at once and
// one block's panel phases overlap the other's trailing update.
template <typename T, int BS>
__global__ void __launch_bounds__(BS, BS == 256 ? 2 : 1)
k_elem_factor_big_b(const DevInst* __restrict__ insts, const int* __restrict__ act, int A,
                    const int* __restrict__ pre_elem, const InstParams* __restrict__ prm,
                    const int* __restrict__ flags, int slab_pb) {
  extern __shared__ unsigned char smraw[];
  for (int t = blockIdx.x; t < pre_elem[A]; t += gridDim.x) {
    const int k = find_item(pre_elem, A, t);
    if (flags[k] & 4) continue;   // condensed by k_elem_factor_rt_b
    const DevInst& I = insts[act[k]];
    const DevFactor<T>& F = inst_factor<T>(I);
    const bool full = (flags[k] & 1) != 0;
    const BigPlace<T> pl = big_place<T>(smraw, F.work, I.P.ext, full);
    // trailing tiles: 8 x 4 (FP32) or 8 x 2 (FP64) within 128 registers per thread
    constexpr int TC = sizeof(T) == 4 ? 4 : 2;
    elem_factor_big<T, 8, TC>(I.P, I.E, I.sigma, prm[k].dw, prm[k].dc, F, t - pre_elem[k], pl,
                              full ? 8 : slab_pb);
  }
}

// FP32: three blocks per SM (more reduction blocks in flight; the levels are
// latency bound), unless WIDE: when the reduction blocks of the batch need so
// much shared memory that one block per SM is all that fits, the kernel is
// compiled for one block per SM and its large blocks get warp-blocked register
// tiles (same arithmetic per entry).
template <typename T, int BT, int WIDE>
__global__ void __launch_bounds__(FBS, (sizeof(T) == 4 && !WIDE) ? 3 : 1)
k_factor_b(const DevInst* __restrict__ insts, const int* __restrict__ act, int A,
           const int* __restrict__ pre_elem, const int* __restrict__ pre_lv, int maxL,
           const int* __restrict__ pre_cs, const InstParams* __restrict__ prm,
           const int* __restrict__ flags, GridBar* gb, size_t smem_bytes, int bcr_full,
           int slab_pb) {
  extern __shared__ unsigned char smraw[];
  unsigned int ep = 0;
  // 1. element condensation: done by k_elem_factor_rt_b / k_elem_factor_big_b
  // before this launch
  // 2. cyclic-reduction levels, then each instance's final block
  for (int lv = 0; lv <= maxL; ++lv) {
    const int* pre = pre_lv + (size_t)lv * (A + 1);
    const bool fin = lv == maxL;
    const int tot = fin ? A : pre[A];
    if constexpr (BT > 0) {
      // instances with flag 8: two blocks of the level per CUDA block
      __shared__ PivotBuf<T> ubh[2];
      __shared__ Pivot<T> pivh[2][RT_MAX_PAIRS];
      __shared__ int cnth[2][3];
      const int half = threadIdx.x >> 7, htid = threadIdx.x & 127;
      const HalfBar hbar{1 + half};
      // each half owns a fixed half of the dynamic shared memory (instances of
      // different sizes may share the block), split into two stage buffers:
      // the next block's inputs are copied into one while the current block
      // is factored from the other
      const size_t hb = (smem_bytes / 2) & ~size_t(15), bb = (hb / 2) & ~size_t(15);
      unsigned char* hbase = smraw + half * hb;
      auto stage_of = [&](int j) { return reinterpret_cast<T*>(hbase + (j & 1) * bb); };
      auto next_rt = [&](int t) {
        for (; t < tot; t += 2 * gridDim.x)
          if (flags[fin ? t : find_item(pre, A, t)] & 8) break;
        return t;
      };
      auto issue = [&](int t, int j) {
        const int k = fin ? t : find_item(pre, A, t);
        const DevInst& I = insts[act[k]];
        bcr_stage_issue<T>(I.P, inst_factor<T>(I), fin ? 1 : 1 << lv, fin ? 1 : 0,
                           fin ? 0 : t - pre[k], htid, stage_of(j));
      };
      int t = next_rt(2 * blockIdx.x + half), j = 0;
      if (t < tot) issue(t, 0);
      while (t < tot) {
        const int tn = next_rt(t + 2 * gridDim.x);
        cp_async_wait_all();
        hbar();
        // the other buffer's last block ended with a half barrier
        if (tn < tot) issue(tn, j + 1);
        const int k = fin ? t : find_item(pre, A, t);
        const DevInst& I = insts[act[k]];
        bcr_factor_staged<T, BT>(I.P, inst_factor<T>(I), fin ? 1 : 1 << lv, fin ? 1 : 0,
                                 fin ? 0 : t - pre[k], htid, hbar, ubh[half].v, stage_of(j),
                                 pivh[half], cnth[half]);
        t = tn;
        ++j;
      }
    }
    // the whole-block pass reuses the shared memory the halves staged in
    if (BT > 0 && bcr_full) __syncthreads();
    for (int t = blockIdx.x; bcr_full && t < tot; t += gridDim.x) {
      const int k = fin ? t : find_item(pre, A, t);
      if (BT > 0 && (flags[k] & 8)) continue;
      const DevInst& I = insts[act[k]];
      const DevFactor<T>& F = inst_factor<T>(I);
      const bool full = (flags[k] & 2) != 0;
      const BigPlace<T> pl = big_place<T>(smraw, F.work, I.P.bext, full);
      const int pb = full ? 8 : slab_pb;
      // trailing tiles: warp-blocked 8 x 4 when the kernel runs one block per
      // SM (WIDE), else the 4 x 4 tiles that fit 80 registers per thread
      constexpr int TR = WIDE ? 8 : 0, TC = WIDE ? 4 : 0;
      if (fin) bcr_factor_big<T, TR, TC>(I.P, F, 1, 1, 0, pl, pb);
      else bcr_factor_big<T, TR, TC>(I.P, F, 1 << lv, 0, t - pre[k], pl, pb);
    }
    grid_barrier(gb, ep);
  }
  // 3. chunk sums of the parameter contributions
  for (int t = blockIdx.x * FBS + threadIdx.x; t < pre_cs[A]; t += gridDim.x * FBS) {
    const int k = find_item(pre_cs, A, t);
    const DevInst& I = insts[act[k]];
    const DevFactor<T>& F = inst_factor<T>(I);
    const int L = I.P.p * I.P.p, G = n_chunks(2 * I.P.N);
    const int it = t - pre_cs[k];
    F.chunkS[it] = chunk_sum_item(F.Scon, 2 * I.P.N, L, G, it / L, it % L);
  }
  grid_barrier(gb, ep);
  // 4. parameter Schur complement, one block per instance
  for (int k = blockIdx.x; k < A; k += gridDim.x) {
    const DevInst& I = insts[act[k]];
    const DevFactor<T>& F = inst_factor<T>(I);
    const size_t need = sizeof(double) * ((size_t)I.P.p * I.P.p + I.P.p);
    double* sS = need <= smem_bytes ? reinterpret_cast<double*>(smraw) : I.S.S;
    schur_block(I.P, F.inert, F.chunkS, I.E.wtt, I.sigma, prm[k].dw, I.S, sS);
    if (threadIdx.x == 0) {
      long long* o = reinterpret_cast<long long*>(I.out + O_INERT);
      o[0] = I.S.inertia[0]; o[1] = I.S.inertia[1]; o[2] = I.S.inertia[2];
    }
  }
  grid_exit(gb);
}

// Batched solve.  Levels below `lsplit` run over the whole grid, a grid
// barrier after each; from level `lsplit` up (few blocks per instance) one
// block owns an instance and separates its levels by block barriers, and the
// same block then solves the parameter system and substitutes back down to
// level `lsplit`.  Every block solve is the same per-warp code as in the
// single-instance launches, so the result does not depend on the split.
template <typename T>
__global__ void __launch_bounds__(FBS)
k_solve_b(const DevInst* __restrict__ insts, const int* __restrict__ act, int A,
          const int* __restrict__ pre_elem, const int* __restrict__ pre_lv, int maxL, int lsplit,
          const int* __restrict__ pre_cs, int ir, int per_warp, GridBar* gb) {
  extern __shared__ unsigned char smraw[];
  unsigned int ep = 0;
  const int warp = threadIdx.x >> 5, wpb = FBS / 32;
  const int gw = blockIdx.x * wpb + warp, nw = gridDim.x * wpb;
  T* wv = reinterpret_cast<T*>(smraw) + (size_t)warp * per_warp;
  auto level_blocks = [&](int lv, int k) {
    const int* pre = pre_lv + (size_t)lv * (A + 1);
    return lv == maxL ? 1 : pre[k + 1] - pre[k];
  };
  for (int t = gw; t < pre_elem[A]; t += nw) {
    const int k = find_item(pre_elem, A, t);
    const DevInst& I = insts[act[k]];
    elem_fwd_one<T>(I.P, inst_factor<T>(I), ir ? I.kr : I.ka, t - pre_elem[k], wv);
  }
  grid_barrier(gb, ep);
  for (int lv = 0; lv < lsplit; ++lv) {
    const int* pre = pre_lv + (size_t)lv * (A + 1);
    for (int t = gw; t < pre[A]; t += nw) {
      const int k = find_item(pre, A, t);
      const DevInst& I = insts[act[k]];
      bcr_fwd_one<T>(I.P, inst_factor<T>(I), 1 << lv, 0, t - pre[k], wv);
    }
    grid_barrier(gb, ep);
  }
  for (int k = blockIdx.x; k < A; k += gridDim.x) {
    const DevInst& I = insts[act[k]];
    for (int lv = lsplit; lv <= maxL; ++lv) {
      const bool fin = lv == maxL;
      const int nb = level_blocks(lv, k);
      for (int bi = warp; bi < nb; bi += wpb)
        bcr_fwd_one<T>(I.P, inst_factor<T>(I), fin ? 1 : 1 << lv, fin ? 1 : 0, bi, wv);
      __syncthreads();
    }
  }
  grid_barrier(gb, ep);
  for (int t = blockIdx.x * FBS + threadIdx.x; t < pre_cs[A]; t += gridDim.x * FBS) {
    const int k = find_item(pre_cs, A, t);
    const DevInst& I = insts[act[k]];
    const DevFactor<T>& F = inst_factor<T>(I);
    const int L = I.P.p, G = n_chunks(2 * I.P.N);
    const int it = t - pre_cs[k];
    F.chunkR[it] = chunk_sum_item(F.Rth, 2 * I.P.N, L, G, it / L, it % L);
  }
  grid_barrier(gb, ep);
  for (int k = blockIdx.x; k < A; k += gridDim.x) {
    const DevInst& I = insts[act[k]];
    double* sol = ir ? I.kc : I.kb;
    // theta_solve_block ends with a block barrier: its shared vector and the
    // per-warp vectors below may overlap
    theta_solve_block(I.P, inst_factor<T>(I).chunkR, ir ? I.kr : I.ka, I.S, sol,
                      reinterpret_cast<double*>(smraw));
    for (int lv = maxL; lv >= lsplit; --lv) {
      const bool fin = lv == maxL;
      const int nb = level_blocks(lv, k);
      for (int bi = warp; bi < nb; bi += wpb)
        bcr_bwd_one<T>(I.P, inst_factor<T>(I), I.S, sol, fin ? 1 : 1 << lv, fin ? 1 : 0, bi, wv);
      __syncthreads();
    }
  }
  grid_barrier(gb, ep);
  for (int lv = lsplit - 1; lv >= 0; --lv) {
    const int* pre = pre_lv + (size_t)lv * (A + 1);
    for (int t = gw; t < pre[A]; t += nw) {
      const int k = find_item(pre, A, t);
      const DevInst& I = insts[act[k]];
      bcr_bwd_one<T>(I.P, inst_factor<T>(I), I.S, ir ? I.kc : I.kb, 1 << lv, 0, t - pre[k], wv);
    }
    grid_barrier(gb, ep);
  }
  for (int t = gw; t < pre_elem[A]; t += nw) {
    const int k = find_item(pre_elem, A, t);
    const DevInst& I = insts[act[k]];
    elem_bwd_one<T>(I.P, inst_factor<T>(I), I.S, ir ? I.kc : I.kb, t - pre_elem[k], wv);
  }
  grid_exit(gb);
}

// ---- host launchers ------------------------------------------------------------------
int bcr_levels(int N) {
  int lv = 0;
  for (int s = 1; s < N; s *= 2) ++lv;
  return lv;
}

// Dynamic shared memory of a panel-eliminated block: everything (full), or
// the panel buffers only when the block is in a global slab (none when they
// are in the slab too).
template <typename T>
static size_t panel_smem(int msz, bool full) {
  const size_t panel = sizeof(T) * big_panel_elems<T>(msz);
  if (full) return panel + sizeof(T) * big_tri_elems(msz);
  return panel_in_global<T>(msz) ? 0 : panel;
}
template <typename T>
size_t elem_factor_smem(const DevProb& P, bool full) { return panel_smem<T>(P.ext, full); }
template <typename T>
size_t bcr_factor_smem(const DevProb& P, bool full) { return panel_smem<T>(P.bext, full); }

// Largest dynamic shared memory of a factorization block.  One limit decides
// both whether a block is factored in shared memory (here and in the batched
// plans) and whether its global slab is allocated; it leaves room for the
// static shared memory of the persistent kernels (< 27 KB) under 227 KB.
constexpr size_t SMEM_LIMIT = FACTOR_SMEM_LIMIT;

template <typename T>
bool elem_uses_smem(const DevProb& P) { return elem_factor_smem<T>(P, true) <= SMEM_LIMIT; }
template <typename T>
bool bcr_uses_smem(const DevProb& P) { return bcr_factor_smem<T>(P, true) <= SMEM_LIMIT; }

// Global workspace (in T elements) needed when a block does not fit in shared memory.
template <typename T>
size_t factor_work_elems(const DevProb& P, int n_slabs) {
  size_t w = 0;
  if (!elem_uses_smem<T>(P)) w = std::max(w, slab_elems<T>(P.ext) * n_slabs);
  if (!bcr_uses_smem<T>(P)) w = std::max(w, slab_elems<T>(P.bext) * n_slabs);
  return w;
}

// cudaFuncAttributeMaxDynamicSharedMemorySize, set only when a launch needs
// more than the kernel's setting so far (per device).
template <typename KernelT>
static void opt_in_smem(KernelT kern, size_t bytes) {
  if (bytes <= SMEM_OPTIN_ABOVE) return;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = done[{dev, (const void*)kern}];
  if (bytes <= cur) return;
  // a kernel that asks for this much shared memory also asks for the largest
  // shared-memory carveout of the SM's L1: by default the driver may pick a
  // smaller one that holds fewer of its blocks
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
          cudaSuccess &&
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) == cudaSuccess)
    cur = bytes;
  else
    cudaGetLastError();
}

template <typename T>
cudaError_t launch_elem_factor(const DevProb& P, const DevEval& E, const double* sigma, double dw,
                               double dc, const DevFactor<T>& F, cudaStream_t st) {
  const int rtn = rt_block_threads<T>(P.ext);
  if (rtn > 0) {
    const size_t sm = elem_stage_bytes<T>(P);
    opt_in_smem(k_elem_factor_rt<T>, sm);
    count_launch();
    k_elem_factor_rt<T><<<P.N, rtn, sm, st>>>(P, E, sigma, dw, dc, F);
    return cudaGetLastError();
  }
  bool es = elem_uses_smem<T>(P);
  size_t sm = elem_factor_smem<T>(P, es);
  if (sm > SMEM_OPTIN_ABOVE)
    cudaFuncSetAttribute(k_elem_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int grid = es ? P.N : std::min(P.N, F.n_slabs);
  count_launch();
  k_elem_factor<T><<<grid, FBS, sm, st>>>(P, E, sigma, dw, dc, F, es ? 1 : 0,
                                           schedule().slab_pairs);
  return cudaGetLastError();
}

template <typename KernelT>
static int coop_grid(KernelT kern, int threads, size_t smem, int want, int reserve = 0) {
  // co-resident blocks per SM per (device, kernel, threads, shared memory),
  // cached: the query costs more host time than a launch.  `reserve` SMs are
  // left out (kernels of another stream hold them), so that the whole grid
  // fits on the others.
  struct Key {
    int dev;
    const void* k;
    int threads;
    size_t smem;
    bool operator<(const Key& o) const {
      return std::tie(dev, k, threads, smem) < std::tie(o.dev, o.k, o.threads, o.smem);
    }
  };
  static std::mutex mu;
  static std::map<Key, std::pair<int, int>> cache;   // (blocks per SM, SMs)
  int dev = 0;
  cudaGetDevice(&dev);
  const Key key{dev, (const void*)kern, threads, smem};
  int per = -1, sms = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) { per = it->second.first; sms = it->second.second; }
  }
  if (per < 0) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = {per, sms};
  }
  const int usable = std::max(1, sms - std::max(0, reserve));
  return std::max(0, std::min(want, per * usable));
}

template <typename T>
cudaError_t launch_factor(const DevProb& P, const DevEval& E, const double* sigma, double dw,
                          double dc, const DevFactor<T>& F, const DevSchur& S, cudaStream_t st) {
  const bool es = elem_uses_smem<T>(P), bs = bcr_uses_smem<T>(P);
  const size_t sme = elem_factor_smem<T>(P, es), smb = bcr_factor_smem<T>(P, bs);
  const size_t sms = sizeof(double) * ((size_t)P.p * P.p + P.p);
  cudaError_t e;
  if ((e = launch_elem_factor<T>(P, E, sigma, dw, dc, F, st)) != cudaSuccess) return e;
  const int bt = bcr_rt_tiles(P.bext);
  auto bcr_level = [&](int s, int fin) -> cudaError_t {
    const int nblk = fin ? 1 : bcr_level_blocks(P.N, s);
    const size_t smr = 2 * sizeof(T) * bcr_stage_elems(P.n, P.p);
    count_launch();
    if (bt == 1 || bt == 2) {
      auto kern = bt == 1 ? k_bcr_factor<T, 1> : k_bcr_factor<T, 2>;
      if (smr > SMEM_OPTIN_ABOVE)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
      kern<<<(nblk + 1) / 2, FBS, smr, st>>>(P, F, s, fin, 1, schedule().slab_pairs);
    } else {
      if (smb > SMEM_OPTIN_ABOVE)
        cudaFuncSetAttribute(k_bcr_factor<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smb);
      const int g = bs ? nblk : std::min(nblk, F.n_slabs);
      k_bcr_factor<T, 0><<<g, FBS, smb, st>>>(P, F, s, fin, bs ? 1 : 0, schedule().slab_pairs);
    }
    return cudaGetLastError();
  };
  for (int s = 1; s < P.N; s *= 2)
    if ((e = bcr_level(s, 0)) != cudaSuccess) return e;
  if ((e = bcr_level(1, 1)) != cudaSuccess) return e;
  // the Schur block works in shared memory up to the factorization limit,
  // otherwise in S.S (p p + p doubles) itself
  const bool sg = sms > SMEM_LIMIT;
  if (!sg && sms > SMEM_OPTIN_ABOVE)
    cudaFuncSetAttribute(k_schur, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms);
  if ((e = launch_chunk_sums(F.Scon, 2 * P.N, P.p * P.p, F.chunkS, st)) != cudaSuccess) return e;
  count_launch();
  k_schur<<<1, SBS, sg ? 0 : sms, st>>>(P, F.inert, F.chunkS, E.wtt, sigma, dw, S, sg ? 1 : 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve(const DevProb& P, const DevFactor<T>& F, const DevSchur& S,
                         const double* b, double* sol, cudaStream_t st) {
  const int tpb = 32 * SOLVE_WARPS;
  cudaError_t e;
  size_t sme = sizeof(T) * (size_t)P.ext * SOLVE_WARPS;
  size_t smb = sizeof(T) * (size_t)P.bext * SOLVE_WARPS;
  if (sme > SMEM_OPTIN_ABOVE) {
    cudaFuncSetAttribute(k_elem_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sme);
    cudaFuncSetAttribute(k_elem_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sme);
  }
  if (smb > SMEM_OPTIN_ABOVE) {
    cudaFuncSetAttribute(k_bcr_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
    cudaFuncSetAttribute(k_bcr_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
  }
  count_launch();
  k_elem_fwd<T><<<ceil_div(P.N, SOLVE_WARPS), tpb, sme, st>>>(P, F, b);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  std::vector<int> strides;
  for (int s = 1; s < P.N; s *= 2) strides.push_back(s);
  for (int s : strides) {
    int nblk = bcr_level_blocks(P.N, s);
    count_launch();
    k_bcr_fwd<T><<<ceil_div(nblk, SOLVE_WARPS), tpb, smb, st>>>(P, F, s, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  count_launch();
  k_bcr_fwd<T><<<1, tpb, smb, st>>>(P, F, 1, 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  size_t smt = sizeof(double) * (size_t)(P.p > 0 ? P.p : 1);
  if ((e = launch_chunk_sums(F.Rth, 2 * P.N, P.p, F.chunkR, st)) != cudaSuccess) return e;
  count_launch();
  k_theta_solve<<<1, SBS, smt, st>>>(P, F.chunkR, b, S, sol);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  count_launch();
  k_bcr_bwd<T><<<1, tpb, smb, st>>>(P, F, S, sol, 1, 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int k = (int)strides.size() - 1; k >= 0; --k) {
    int s = strides[k];
    int nblk = bcr_level_blocks(P.N, s);
    count_launch();
    k_bcr_bwd<T><<<ceil_div(nblk, SOLVE_WARPS), tpb, smb, st>>>(P, F, S, sol, s, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  count_launch();
  k_elem_bwd<T><<<ceil_div(P.N, SOLVE_WARPS), tpb, sme, st>>>(P, F, S, sol);
  return cudaGetLastError();
}

// Batched launchers.  `grid_cap` limits the grid when some instance uses its
// global slabs (at most n_slabs blocks may run).  Factorization parts: 1 the
// register-tiled element kernel, 4 the large-element kernel, 2 the rest (cyclic
// reduction and parameter Schur complement in the cooperative kernel).
template <typename T>
cudaError_t launch_factor_b(const DevInst* insts, const int* act, int A, const int* pre_elem,
                            const int* pre_lv, int maxL, const int* pre_cs,
                            const InstParams* prm, const int* flags, GridBar* gb, size_t smem,
                            int grid_cap, int rt_threads, size_t rt_smem, int tot_elem,
                            int big_grid, size_t big_smem, int bcr_tpt, int bcr_full, int parts,
                            cudaStream_t st, int reserve) {
  if (A == 0) return cudaSuccess;
  if ((parts & 1) && rt_threads > 0 && tot_elem > 0) {
    if (rt_threads > RT_MAX_THREADS) return cudaErrorInvalidValue;
    opt_in_smem(k_elem_factor_rt_b<T>, rt_smem);
    count_launch();
    k_elem_factor_rt_b<T><<<tot_elem, rt_threads, rt_smem, st>>>(insts, act, A, pre_elem, prm,
                                                                 flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const Schedule sch = schedule();
  if ((parts & 4) && big_grid > 0) {
    count_launch();
    if (sch.big_threads == 256) {
      opt_in_smem(k_elem_factor_big_b<T, 256>, big_smem);
      k_elem_factor_big_b<T, 256><<<big_grid, 256, big_smem, st>>>(insts, act, A, pre_elem, prm,
                                                                   flags, sch.slab_pairs);
    } else {
      opt_in_smem(k_elem_factor_big_b<T, 512>, big_smem);
      k_elem_factor_big_b<T, 512><<<big_grid, 512, big_smem, st>>>(insts, act, A, pre_elem, prm,
                                                                   flags, sch.slab_pairs);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (!(parts & 2)) return cudaSuccess;
  // one block per SM is all that fits when smem exceeds a third of an SM's
  // shared memory: then the kernel variant compiled for one block per SM
  int dev = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const bool wide = sizeof(T) == 4 && bcr_full && 3 * (smem + 1024) > (size_t)smem_sm;
  auto kern = wide ? (bcr_tpt == 1 ? k_factor_b<T, 1, 1>
                      : bcr_tpt == 2 ? k_factor_b<T, 2, 1> : k_factor_b<T, 0, 1>)
                   : (bcr_tpt == 1 ? k_factor_b<T, 1, 0>
                      : bcr_tpt == 2 ? k_factor_b<T, 2, 0> : k_factor_b<T, 0, 0>);
  opt_in_smem(kern, smem);
  int grid = coop_grid(kern, FBS, smem, grid_cap, reserve);
  if (grid < 1) return cudaErrorInvalidConfiguration;
  int slab_pb = sch.slab_pairs;
  void* args[] = {(void*)&insts, (void*)&act, &A, (void*)&pre_elem, (void*)&pre_lv, &maxL,
                  (void*)&pre_cs, (void*)&prm, (void*)&flags, &gb, &smem, &bcr_full, &slab_pb};
  count_launch();
  return cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(FBS), args, smem, st);
}

template <typename T>
cudaError_t launch_solve_b(const DevInst* insts, const int* act, int A, const int* pre_elem,
                           const int* pre_lv, int maxL, int lsplit, const int* pre_cs, int ir,
                           int per_warp,
                           GridBar* gb, int max_p, int grid_want, cudaStream_t st, int reserve) {
  if (A == 0) return cudaSuccess;
  size_t smem = std::max(sizeof(T) * (size_t)per_warp * (FBS / 32),
                         sizeof(double) * (size_t)std::max(max_p, 1));
  opt_in_smem(k_solve_b<T>, smem);
  int grid = coop_grid(k_solve_b<T>, FBS, smem, grid_want, reserve);
  if (grid < 1) return cudaErrorInvalidConfiguration;
  void* args[] = {(void*)&insts, (void*)&act, &A, (void*)&pre_elem, (void*)&pre_lv, &maxL,
                  &lsplit, (void*)&pre_cs, &ir, &per_warp, &gb};
  count_launch();
  return cudaLaunchCooperativeKernel((void*)k_solve_b<T>, dim3(grid), dim3(FBS), args, smem, st);
}

template cudaError_t launch_factor_b<float>(const DevInst*, const int*, int, const int*,
                                            const int*, int, const int*, const InstParams*,
                                            const int*, GridBar*, size_t, int, int, size_t, int,
                                            int, size_t, int, int, int, cudaStream_t, int);
template cudaError_t launch_factor_b<double>(const DevInst*, const int*, int, const int*,
                                             const int*, int, const int*, const InstParams*,
                                             const int*, GridBar*, size_t, int, int, size_t, int,
                                             int, size_t, int, int, int, cudaStream_t, int);
int bcr_rt_tiles_of(const DevProb& P) { return bcr_rt_tiles(P.bext); }
size_t elem_rt_stage_bytes(const DevProb& P, bool f32) {
  return f32 ? elem_stage_bytes<float>(P) : elem_stage_bytes<double>(P);
}
size_t bcr_rt_stage_bytes(const DevProb& P, bool f32) {
  const size_t one = (f32 ? sizeof(float) : sizeof(double)) * bcr_stage_elems(P.n, P.p);
  return 4 * ((one + 15) & ~size_t(15));   // two halves, two stage buffers each
}
int elem_rt_threads(const DevProb& P, bool f32) {
  return f32 ? rt_block_threads<float>(P.ext) : rt_block_threads<double>(P.ext);
}
template cudaError_t launch_solve_b<float>(const DevInst*, const int*, int, const int*, const int*,
                                           int, int, const int*, int, int, GridBar*, int, int,
                                           cudaStream_t, int);
template cudaError_t launch_solve_b<double>(const DevInst*, const int*, int, const int*,
                                            const int*, int, int, const int*, int, int, GridBar*,
                                            int, int, cudaStream_t, int);
template size_t elem_factor_smem<float>(const DevProb&, bool);
template size_t elem_factor_smem<double>(const DevProb&, bool);
template size_t bcr_factor_smem<float>(const DevProb&, bool);
template size_t bcr_factor_smem<double>(const DevProb&, bool);

template cudaError_t launch_factor<double>(const DevProb&, const DevEval&, const double*, double,
                                           double, const DevFactor<double>&, const DevSchur&,
                                           cudaStream_t);
template cudaError_t launch_factor<float>(const DevProb&, const DevEval&, const double*, double,
                                          double, const DevFactor<float>&, const DevSchur&,
                                          cudaStream_t);
template cudaError_t launch_solve<double>(const DevProb&, const DevFactor<double>&,
                                          const DevSchur&, const double*, double*, cudaStream_t);
template cudaError_t launch_solve<float>(const DevProb&, const DevFactor<float>&,
                                         const DevSchur&, const double*, double*, cudaStream_t);
template cudaError_t launch_elem_factor<double>(const DevProb&, const DevEval&, const double*,
                                                double, double, const DevFactor<double>&,
                                                cudaStream_t);
template cudaError_t launch_elem_factor<float>(const DevProb&, const DevEval&, const double*,
                                               double, double, const DevFactor<float>&,
                                               cudaStream_t);
template size_t factor_work_elems<double>(const DevProb&, int);
template size_t factor_work_elems<float>(const DevProb&, int);

}  // namespace collo
