// Batched execution of the hot path: a Runner holds the device descriptors of
// up to `capacity` problems and launches every phase of the Newton step for a
// set of active problems at once (one grid over all their elements, one
// cooperative kernel for all their factorizations / solves).  A single
// problem is a batch of one.  On top of it sit the lock-step batched
// interior-point driver (collo_ipm_solve, collo_batch_solve) and the
// continuous-batching server (collo_server_*).
//
// Results of a problem do not depend on the other members of its batch: every
// kernel computes an instance's values from that instance's data only, each
// element / reduction block in a fixed order, so a problem solved alone and in
// a mix follows the same arithmetic.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include <cstdlib>

#include "problem.cuh"

namespace collo {

constexpr int OUTS = 32;                  // doubles of DevInst::out per instance
constexpr size_t KSMEM_LIMIT = FACTOR_SMEM_LIMIT;

// Relative KKT residual above which refinement from an FP32 factorization
// counts as failed (the step is then redone with an FP64 factorization).
constexpr double ESCALATE_REL = 1e-6;

// ---- plans ---------------------------------------------------------------------------
struct Plan {
  std::vector<int> slots;
  int A = 0, maxL = 0, tot_elem = 0, max_p = 0, max_n = 0;   // max_n: most state rows of an element, (K + 1) n
  int lsplit = 0;   // first reduction level the solve runs one block per instance
  long long tot_upd = 0;
  int* d_int = nullptr; int* h_int = nullptr; size_t cap_int = 0;
  long long* d_ll = nullptr; long long* h_ll = nullptr; size_t cap_ll = 0;
  InstParams* d_prm = nullptr; InstParams* h_prm = nullptr; size_t cap_prm = 0;
  cudaEvent_t ev_int = nullptr, ev_prm = nullptr;
  bool int_pending = false, prm_pending = false;
  size_t off_act = 0, off_elem = 0, off_lv = 0, off_cs_s = 0, off_cs_r = 0, off_f32 = 0,
         off_f64 = 0, off_sw_w = 0, off_sw_c = 0;
  int n_sw_w = 0, n_sw_c = 0;
  size_t smem_eval = 0, smem_f[2] = {0, 0}, smem_sw_w = 0, smem_sw_c = 0;
  int cap_f[2] = {1 << 30, 1 << 30};
  int per_warp[2] = {0, 0};
  int rt_threads[2] = {0, 0};   // block size of the register-tiled element kernel
  size_t rt_smem[2] = {0, 0};   // its dynamic shared memory
  int big_grid[2] = {0, 0};     // grid of the large-element kernel (0: no such element)
  size_t big_smem[2] = {0, 0};  // its dynamic shared memory
  int bcr_tpt = 0;          // ... of the register-tiled cyclic-reduction blocks
  int bcr_full = 0;         // some instance's reduction blocks use the whole-block path

  const int* act() const { return d_int + off_act; }
  const int* pre_elem() const { return d_int + off_elem; }
  const int* pre_lv() const { return d_int + off_lv; }
  const int* pre_cs_s() const { return d_int + off_cs_s; }
  const int* pre_cs_r() const { return d_int + off_cs_r; }
  const int* flags(int prec) const { return d_int + (prec ? off_f32 : off_f64); }
  const long long* pre_upd() const { return d_ll; }

  ~Plan() {
    if (d_int) cudaFree(d_int);
    if (h_int) cudaFreeHost(h_int);
    if (d_ll) cudaFree(d_ll);
    if (h_ll) cudaFreeHost(h_ll);
    if (d_prm) cudaFree(d_prm);
    if (h_prm) cudaFreeHost(h_prm);
    if (ev_int) cudaEventDestroy(ev_int);
    if (ev_prm) cudaEventDestroy(ev_prm);
  }
};

template <typename T>
static cudaError_t grow(T** d, T** h, size_t* cap, size_t need) {
  if (need <= *cap) return cudaSuccess;
  if (*d) cudaFree(*d);
  if (*h) cudaFreeHost(*h);
  *d = nullptr; *h = nullptr;
  size_t c = std::max<size_t>(need, 2 * *cap);
  cudaError_t e = cudaMalloc((void**)d, c * sizeof(T));
  if (e != cudaSuccess) return e;
  e = cudaMallocHost((void**)h, c * sizeof(T));
  if (e != cudaSuccess) return e;
  *cap = c;
  return cudaSuccess;
}

struct Runner {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int capacity = 0;
  int* h_err = nullptr;        // pinned copy of the grid-barrier error flag
  bool err_fresh = false;      // h_err read after the last launch
  DevInst* d_insts = nullptr;
  std::vector<DevInst> h_insts;
  std::vector<collo_problem*> probs;
  double* d_outs = nullptr;
  double* h_outs = nullptr;
  GridBar* gbar = nullptr;
  // 0: all active, 1: subset, 2: sub-subset (precision split), 3: scratch,
  // 4: forward sweeps of the server's admissions on its side stream
  Plan plans[5];
  // SMs the cooperative factorization and solve grids leave free for the
  // server's forward sweeps running on its side stream
  int reserve_sms = 0;

  ~Runner() {
    if (d_insts) cudaFree(d_insts);
    if (d_outs) cudaFree(d_outs);
    if (h_outs) cudaFreeHost(h_outs);
    if (h_err) cudaFreeHost(h_err);
    if (gbar) cudaFree(gbar);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  collo_status init(int cap, int dev, cudaStream_t st) {
    capacity = cap;
    device = dev;
    if (st) { stream = st; } else {
      COLLO_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
      own_stream = true;
    }
    // slots [0, cap) hold the problems, [cap, 2 cap) their shadows (spare
    // factorization storage for speculative inertia correction)
    COLLO_CUDA(cudaMalloc(&d_insts, sizeof(DevInst) * 2 * cap));
    COLLO_CUDA(cudaMalloc(&d_outs, sizeof(double) * OUTS * 2 * cap));
    COLLO_CUDA(cudaMemset(d_outs, 0, sizeof(double) * OUTS * 2 * cap));
    COLLO_CUDA(cudaMallocHost(&h_outs, sizeof(double) * OUTS * 2 * cap));
    COLLO_CUDA(cudaMallocHost(&h_err, sizeof(int)));
    *h_err = 0;
    COLLO_CUDA(cudaMalloc(&gbar, sizeof(GridBar)));
    COLLO_CUDA(cudaMemset(gbar, 0, sizeof(GridBar)));
    h_insts.assign(2 * cap, DevInst{});
    probs.assign(2 * cap, nullptr);
    for (auto& pl : plans) {
      COLLO_CUDA(cudaEventCreateWithFlags(&pl.ev_int, cudaEventDisableTiming));
      COLLO_CUDA(cudaEventCreateWithFlags(&pl.ev_prm, cudaEventDisableTiming));
    }
    return COLLO_OK;
  }

  // Place problem pr in slot s (its descriptor, with out pointing into d_outs),
  // and its shadow in slot capacity + s: the same problem with the spare
  // factorization and Schur storage.
  collo_status attach(int s, collo_problem* pr) {
    DevInst I = pr->inst;
    I.F32 = pr->f32.F;
    I.F64 = pr->f64.F;
    I.out = d_outs + (size_t)s * OUTS;
    h_insts[s] = I;
    probs[s] = pr;
    const int sh = shadow(s);
    I.F32 = pr->f32_spare.F;
    I.F64 = pr->f64_spare.F;
    I.S = pr->S_spare;
    if (pr->c_spare) {   // a second line-search trial evaluates into these
      I.E.c = pr->c_spare;
      I.E.part = pr->part_spare;
      I.E.red = pr->red_spare;
    }
    I.out = d_outs + (size_t)sh * OUTS;
    h_insts[sh] = I;
    probs[sh] = pr;
    COLLO_CUDA(cudaMemcpyAsync(d_insts + s, &h_insts[s], sizeof(DevInst), cudaMemcpyHostToDevice,
                               stream));
    COLLO_CUDA(cudaMemcpyAsync(d_insts + sh, &h_insts[sh], sizeof(DevInst),
                               cudaMemcpyHostToDevice, stream));
    COLLO_CUDA(cudaStreamSynchronize(stream));
    return COLLO_OK;
  }
  int shadow(int s) const { return capacity + s; }

  // Wait settings of the persistent kernels' grid barrier (see GridBar).
  collo_status set_wait(long long polls, int unreachable) {
    GridBar g{};
    g.extra = unreachable ? 1u : 0u;
    g.spin_limit = polls > 0 ? polls : 0;
    COLLO_CUDA(cudaStreamSynchronize(stream));
    COLLO_CUDA(cudaMemcpy(&gbar->extra, &g.extra, sizeof(g.extra), cudaMemcpyHostToDevice));
    COLLO_CUDA(cudaMemcpy(&gbar->spin_limit, &g.spin_limit, sizeof(g.spin_limit),
                          cudaMemcpyHostToDevice));
    return COLLO_OK;
  }

  const DevProb& P(int s) const { return h_insts[s].P; }
  double* out(int s) { return h_outs + (size_t)s * OUTS; }

  // Build plan `which` for the given slots and upload it.
  collo_status set_plan(int which, const std::vector<int>& slots) {
    Plan& pl = plans[which];
    if (pl.int_pending) { cudaEventSynchronize(pl.ev_int); pl.int_pending = false; }
    const int A = (int)slots.size();
    pl.slots = slots;
    pl.A = A;
    int maxL = 0, maxp = 0;
    for (int s : slots) {
      int lv = 0;
      for (int st = 1; st < P(s).N; st *= 2) ++lv;
      maxL = std::max(maxL, lv);
      maxp = std::max(maxp, P(s).p);
    }
    pl.maxL = maxL;
    pl.max_p = maxp;
    pl.max_n = 0;
    for (int s : slots) pl.max_n = std::max(pl.max_n, P(s).np * P(s).n);
    const size_t n_int = (size_t)A + (A + 1) * (size_t)(4 + maxL + 1) + 2 * (size_t)A + 2 * (size_t)A;
    cudaError_t e = grow(&pl.d_int, &pl.h_int, &pl.cap_int, n_int);
    if (e == cudaSuccess) e = grow(&pl.d_ll, &pl.h_ll, &pl.cap_ll, (size_t)A + 1);
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return COLLO_ERR_OOM; }
    int* h = pl.h_int;
    size_t o = 0;
    pl.off_act = o; for (int k = 0; k < A; ++k) h[o + k] = slots[k]; o += A;
    pl.off_elem = o; h[o] = 0;
    for (int k = 0; k < A; ++k) h[o + k + 1] = h[o + k] + P(slots[k]).N;
    pl.tot_elem = h[o + A]; o += A + 1;
    pl.off_lv = o;
    pl.lsplit = maxL;
    for (int lv = maxL; lv >= 0; --lv) {
      int most = 0;
      for (int k = 0; k < A; ++k) {
        const int N = P(slots[k]).N, st = 1 << lv;
        most = std::max(most, (lv < maxL && N > st) ? (N - st + 2 * st - 1) / (2 * st) : 0);
      }
      if (most > schedule().solve_top) break;
      pl.lsplit = lv;
    }
    for (int lv = 0; lv <= maxL; ++lv) {
      h[o] = 0;
      for (int k = 0; k < A; ++k) {
        const int N = P(slots[k]).N, st = 1 << lv;
        const int cnt = (lv < maxL && N > st) ? (N - st + 2 * st - 1) / (2 * st) : 0;
        h[o + k + 1] = h[o + k] + cnt;
      }
      o += A + 1;
    }
    pl.off_cs_s = o; h[o] = 0;
    for (int k = 0; k < A; ++k) {
      const DevProb& Q = P(slots[k]);
      h[o + k + 1] = h[o + k] + n_chunks(2 * Q.N) * Q.p * Q.p;
    }
    o += A + 1;
    pl.off_cs_r = o; h[o] = 0;
    for (int k = 0; k < A; ++k) {
      const DevProb& Q = P(slots[k]);
      h[o + k + 1] = h[o + k] + n_chunks(2 * Q.N) * Q.p;
    }
    o += A + 1;
    // per-precision smem flags, kernel smem sizes and grid caps
    for (int prec = 0; prec < 2; ++prec) {
      const bool f32 = prec == 1;
      const size_t off = o;
      size_t smem = 0;
      int cap = 1 << 30, pw = 0, tpt = 0, btpt = 0, bfull = 0;
      size_t rts = 0, bsm = 0;
      int bcap = 1 << 30, nbig = 0;
      for (int k = 0; k < A; ++k) {
        const DevProb& Q = P(slots[k]);
        const size_t se = f32 ? elem_factor_smem<float>(Q, true) : elem_factor_smem<double>(Q, true);
        const size_t sb = f32 ? bcr_factor_smem<float>(Q, true) : bcr_factor_smem<double>(Q, true);
        const size_t ve = f32 ? elem_factor_smem<float>(Q, false) : elem_factor_smem<double>(Q, false);
        const size_t vb = f32 ? bcr_factor_smem<float>(Q, false) : bcr_factor_smem<double>(Q, false);
        const int rt = elem_rt_threads(Q, f32), brt = bcr_rt_tiles_of(Q);
        int fl = 0;
        size_t need = 0;
        if (rt > 0) {                  // elements condensed by the register-tiled kernel
          fl |= 1 | 4;
          tpt = std::max(tpt, rt);
          rts = std::max(rts, elem_rt_stage_bytes(Q, f32));
        } else {                       // ... or by the large-element kernel
          if (se <= KSMEM_LIMIT) { fl |= 1; bsm = std::max(bsm, se); }
          else { bsm = std::max(bsm, ve); bcap = std::min(bcap, probs[slots[k]]->n_slabs); }
          nbig += Q.N;
        }
        if (brt > 0) {                 // register-tiled reduction blocks
          fl |= 2 | 8;
          btpt = std::max(btpt, brt);
          need = std::max(need, bcr_rt_stage_bytes(Q, f32));
        } else {
          bfull = 1;
          need = std::max(need, vb);
          if (sb <= KSMEM_LIMIT) { fl |= 2; need = std::max(need, sb); }
        }
        const size_t ss = sizeof(double) * ((size_t)Q.p * Q.p + Q.p);
        if (ss <= KSMEM_LIMIT) need = std::max(need, ss);
        // the cooperative kernel uses a global slab only for reduction blocks
        if (!(fl & 2)) cap = std::min(cap, probs[slots[k]]->n_slabs);
        smem = std::max(smem, need);
        h[off + k] = fl;
        pw = std::max(pw, std::max(Q.ext, Q.bext));
      }
      o += A;
      if (f32) pl.off_f32 = off; else pl.off_f64 = off;
      pl.smem_f[prec] = smem;
      pl.cap_f[prec] = cap;
      pl.per_warp[prec] = pw;
      pl.rt_threads[prec] = tpt;
      pl.rt_smem[prec] = rts;
      pl.big_grid[prec] = nbig > 0 ? std::min(bcap, pl.tot_elem) : 0;
      pl.big_smem[prec] = bsm;
      pl.bcr_tpt = btpt;
      pl.bcr_full = bfull;
    }
    // forward-sweep lists and eval shared memory
    pl.off_sw_w = o;
    pl.n_sw_w = 0; pl.smem_sw_w = 0;
    for (int k = 0; k < A; ++k)
      if (P(slots[k]).K * P(slots[k]).n <= 32) {
        h[o + pl.n_sw_w++] = slots[k];
        pl.smem_sw_w = std::max(pl.smem_sw_w, sweep_warp_smem_bytes(P(slots[k])));
      }
    o += A;
    pl.off_sw_c = o;
    pl.n_sw_c = 0; pl.smem_sw_c = 0;
    for (int k = 0; k < A; ++k)
      if (P(slots[k]).K * P(slots[k]).n > 32) {
        h[o + pl.n_sw_c++] = slots[k];
        pl.smem_sw_c = std::max(pl.smem_sw_c,
                                sweep_smem_bytes(P(slots[k]), probs[slots[k]]->sweep_work == nullptr));
      }
    o += A;
    pl.smem_eval = 0;
    for (int k = 0; k < A; ++k) pl.smem_eval = std::max(pl.smem_eval, eval_smem_bytes(P(slots[k])));
    pl.h_ll[0] = 0;
    for (int k = 0; k < A; ++k)
      pl.h_ll[k + 1] = pl.h_ll[k] + h_insts[slots[k]].n_x + h_insts[slots[k]].n_c;
    pl.tot_upd = pl.h_ll[A];
    COLLO_CUDA(cudaMemcpyAsync(pl.d_int, pl.h_int, o * sizeof(int), cudaMemcpyHostToDevice, stream));
    COLLO_CUDA(cudaMemcpyAsync(pl.d_ll, pl.h_ll, (A + 1) * sizeof(long long),
                               cudaMemcpyHostToDevice, stream));
    COLLO_CUDA(cudaEventRecord(pl.ev_int, stream));
    pl.int_pending = true;
    return COLLO_OK;
  }

  // Upload per-instance parameters of plan `which` (fill() writes h_prm[k]).
  template <typename Fill>
  collo_status set_params(int which, Fill fill) {
    Plan& pl = plans[which];
    if (pl.prm_pending) { cudaEventSynchronize(pl.ev_prm); pl.prm_pending = false; }
    cudaError_t e = grow(&pl.d_prm, &pl.h_prm, &pl.cap_prm, (size_t)std::max(pl.A, 1));
    if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return COLLO_ERR_OOM; }
    for (int k = 0; k < pl.A; ++k) {
      InstParams ip{};
      ip.obj_factor = 1.0;
      ip.ksig = 1e10;
      fill(k, pl.slots[k], ip);
      pl.h_prm[k] = ip;
    }
    COLLO_CUDA(cudaMemcpyAsync(pl.d_prm, pl.h_prm, sizeof(InstParams) * std::max(pl.A, 1),
                               cudaMemcpyHostToDevice, stream));
    COLLO_CUDA(cudaEventRecord(pl.ev_prm, stream));
    pl.prm_pending = true;
    return COLLO_OK;
  }

  // Copy the per-instance outputs to the host and wait.
  collo_status read_outs() {
    COLLO_CUDA(cudaMemcpyAsync(h_outs, d_outs, sizeof(double) * OUTS * 2 * capacity,
                               cudaMemcpyDeviceToHost, stream));
    COLLO_CUDA(cudaMemcpyAsync(h_err, &gbar->err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    COLLO_CUDA(cudaStreamSynchronize(stream));
    err_fresh = true;
    for (auto& pl : plans) { pl.int_pending = false; pl.prm_pending = false; }
    return COLLO_OK;
  }

  // Grid-barrier error of the persistent kernels launched so far (read with the
  // last read_outs when nothing was launched since; otherwise read now).
  collo_status check_barrier() {
    if (!err_fresh) {
      COLLO_CUDA(cudaMemcpyAsync(h_err, &gbar->err, sizeof(int), cudaMemcpyDeviceToHost, stream));
      COLLO_CUDA(cudaStreamSynchronize(stream));
    }
    err_fresh = false;
    const int err = *h_err;
    if (err) {
      cudaMemsetAsync(&gbar->err, 0, sizeof(int), stream);
      set_error("grid barrier of a persistent kernel timed out");
      return COLLO_ERR_TIMEOUT;
    }
    return COLLO_OK;
  }

  // ---- phases on plan `which` ----------------------------------------------------
  collo_status eval(int which, int xsel, int dxsel, int lsel, bool deriv) {
    Plan& pl = plans[which];
    COLLO_CUDA(launch_eval_b(d_insts, pl.act(), pl.A, pl.pre_elem(), pl.tot_elem, pl.d_prm, xsel,
                             dxsel, lsel, deriv, pl.smem_eval, stream));
    return COLLO_OK;
  }
  collo_status resid(int which, int mode) {
    Plan& pl = plans[which];
    COLLO_CUDA(launch_resid_b(d_insts, pl.act(), pl.A, pl.pre_elem(), pl.tot_elem, pl.max_n,
                              pl.d_prm, mode, stream));
    return COLLO_OK;
  }
  // parts: 1 register-tiled element condensation, 4 large-element condensation,
  // 2 the rest (cyclic reduction, parameter Schur complement); 7 all
  collo_status factor(int which, int prec, int parts = 7) {
    Plan& pl = plans[which];
    err_fresh = false;
    {
      // a block factored outside shared memory needs its global slab
      const int p = prec == COLLO_PRECISION_MIXED ? 1 : 0;
      const int* fl = pl.h_int + (p ? pl.off_f32 : pl.off_f64);
      for (int k = 0; k < pl.A; ++k) {
        const DevInst& I = h_insts[pl.slots[k]];
        const bool slab = (fl[k] & 3) != 3;
        const bool has = p ? I.F32.work != nullptr : I.F64.work != nullptr;
        if (slab && !has) {
          set_error("internal: factorization block needs a global slab that was not allocated");
          return COLLO_ERR_DEVICE;
        }
      }
    }
    cudaError_t e;
    const int p = prec == COLLO_PRECISION_MIXED ? 1 : 0;
    if (p)
      e = launch_factor_b<float>(d_insts, pl.act(), pl.A, pl.pre_elem(), pl.pre_lv(), pl.maxL,
                                 pl.pre_cs_s(), pl.d_prm, pl.flags(1), gbar, pl.smem_f[1],
                                 std::min(pl.cap_f[1], std::max(pl.tot_elem, pl.A)),
                                 pl.rt_threads[1], pl.rt_smem[1], pl.tot_elem, pl.big_grid[1],
                                 pl.big_smem[1], pl.bcr_tpt, pl.bcr_full, parts, stream,
                                 reserve_sms);
    else
      e = launch_factor_b<double>(d_insts, pl.act(), pl.A, pl.pre_elem(), pl.pre_lv(), pl.maxL,
                                  pl.pre_cs_s(), pl.d_prm, pl.flags(0), gbar, pl.smem_f[0],
                                  std::min(pl.cap_f[0], std::max(pl.tot_elem, pl.A)),
                                  pl.rt_threads[0], pl.rt_smem[0], pl.tot_elem, pl.big_grid[0],
                                  pl.big_smem[0], pl.bcr_tpt, pl.bcr_full, parts, stream,
                                  reserve_sms);
    COLLO_CUDA(e);
    return COLLO_OK;
  }
  collo_status solve(int which, int prec, int ir) {
    Plan& pl = plans[which];
    err_fresh = false;
    cudaError_t e;
    const int per = std::max(1, schedule().solve_elems);
    const int want = std::max(pl.A, (pl.tot_elem + per - 1) / per);
    if (prec == COLLO_PRECISION_MIXED)
      e = launch_solve_b<float>(d_insts, pl.act(), pl.A, pl.pre_elem(), pl.pre_lv(), pl.maxL, pl.lsplit,
                                pl.pre_cs_r(), ir, pl.per_warp[1], gbar, pl.max_p, want, stream,
                                reserve_sms);
    else
      e = launch_solve_b<double>(d_insts, pl.act(), pl.A, pl.pre_elem(), pl.pre_lv(), pl.maxL, pl.lsplit,
                                 pl.pre_cs_r(), ir, pl.per_warp[0], gbar, pl.max_p, want, stream,
                                 reserve_sms);
    COLLO_CUDA(e);
    return COLLO_OK;
  }
  collo_status update(int which, int mode) {
    Plan& pl = plans[which];
    COLLO_CUDA(launch_update_b(d_insts, pl.act(), pl.A, pl.pre_upd(), pl.tot_upd, pl.d_prm, mode,
                               stream));
    return COLLO_OK;
  }
};

// Problem-owned runner for the single-instance API.
collo_status self_runner(collo_problem* pr, Runner** out) {
  if (!pr->self) {
    Runner* r = new Runner();
    collo_status s = r->init(1, pr->device, pr->stream);
    if (s == COLLO_OK && (pr->wait_polls > 0 || pr->wait_unreachable))
      s = r->set_wait(pr->wait_polls, pr->wait_unreachable);
    if (s != COLLO_OK) { delete r; return s; }
    pr->self = r;
  }
  *out = pr->self;
  return COLLO_OK;
}

// (Re)attach a problem to its own runner, e.g. after factor storage grew.
collo_status self_attach(collo_problem* pr, Runner** out) {
  collo_status s = self_runner(pr, out);
  if (s != COLLO_OK) return s;
  return (*out)->attach(0, pr);
}

// ---- refinement: solve for the rhs in ka (plan which), refine into kb ----------------
// Returns per-instance relative residuals in rel[] (indexed like the plan).
static collo_status solve_refine(Runner& R, int which, const std::vector<int>& prec_of_slot,
                                 const std::vector<double>& dw, const std::vector<double>& dc,
                                 int refine_max, double refine_tol, std::vector<int>& sweeps,
                                 std::vector<double>& rel) {
  Plan& pl = R.plans[which];
  const std::vector<int> all = pl.slots;
  const int A = (int)all.size();
  sweeps.assign(A, 0);
  rel.assign(A, 0.0);
  std::map<int, int> pos;
  for (int k = 0; k < A; ++k) pos[all[k]] = k;
  // initial solve per precision group
  std::vector<int> groups[2];
  for (int s : all) groups[prec_of_slot[s] == COLLO_PRECISION_MIXED ? 1 : 0].push_back(s);
  for (int g = 0; g < 2; ++g) {
    if (groups[g].empty()) continue;
    collo_status st = R.set_plan(2, groups[g]);
    if (st != COLLO_OK) return st;
    st = R.solve(2, g ? COLLO_PRECISION_MIXED : COLLO_PRECISION_FP64, 0);
    if (st != COLLO_OK) return st;
  }
  std::vector<int> todo = all;
  for (int sweep = 0;; ++sweep) {
    collo_status st = R.set_plan(1, todo);
    if (st != COLLO_OK) return st;
    st = R.set_params(1, [&](int, int s, InstParams& ip) { ip.dw = dw[pos[s]]; ip.dc = dc[pos[s]]; });
    if (st != COLLO_OK) return st;
    st = R.resid(1, 2 /* R_IR */);
    if (st != COLLO_OK) return st;
    st = R.read_outs();
    if (st != COLLO_OK) return st;
    st = R.check_barrier();
    if (st != COLLO_OK) return st;
    std::vector<int> next;
    for (int s : todo) {
      const double* o = R.out(s);
      const double rn = std::max(o[O_RX], o[O_RC]);
      const double r = rn / std::max(1.0, o[O_BMAX]);
      const double prev = rel[pos[s]];
      rel[pos[s]] = r;
      // an FP32-factor refinement above ESCALATE_REL that no longer halves its
      // residual per sweep ends as a failure (the step is redone in FP64):
      // stop it now instead of after refine_max sweeps
      const bool stalled = prec_of_slot[s] == COLLO_PRECISION_MIXED && sweeps[pos[s]] >= 2 &&
                           r > ESCALATE_REL && r > 0.5 * prev;
      if (r > refine_tol && sweeps[pos[s]] < refine_max && std::isfinite(r) && !stalled)
        next.push_back(s);
    }
    if (next.empty()) break;
    for (int s : next) sweeps[pos[s]]++;
    std::vector<int> gr[2];
    for (int s : next) gr[prec_of_slot[s] == COLLO_PRECISION_MIXED ? 1 : 0].push_back(s);
    for (int g = 0; g < 2; ++g) {
      if (gr[g].empty()) continue;
      st = R.set_plan(2, gr[g]);
      if (st != COLLO_OK) return st;
      st = R.solve(2, g ? COLLO_PRECISION_MIXED : COLLO_PRECISION_FP64, 1);
      if (st != COLLO_OK) return st;
      st = R.update(2, 1 /* kb += kc */);
      if (st != COLLO_OK) return st;
    }
    todo = next;
  }
  return COLLO_OK;
}

// ---- the batched interior-point driver --------------------------------------------
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

static Opt make_opt(const collo_ipm_options* opts) {
  collo_ipm_options uo;
  if (opts) uo = *opts; else collo_ipm_options_default(&uo);
  Opt o;
  o.tol = uo.tol; o.acc_tol = uo.acceptable_tol; o.acc_iter = uo.acceptable_iter;
  o.max_iter = uo.max_iter; o.max_wall = uo.max_wall_time; o.precision = uo.precision;
  o.mixed_mu_switch = uo.mixed_mu_switch; o.refine_max = uo.refine_max;
  o.refine_tol = uo.refine_tol; o.verbose = uo.verbose;
  return o;
}

enum { RUNNING = 1000 };

// ---- optional phase profile of the iteration driver (COLLO_PROFILE=1) --------------
// Host wall time per phase of ipm_iteration, with a stream synchronisation at
// each phase boundary (only when enabled), and counts of the rounds of the
// phases that loop over shrinking subsets.
enum ProfPhase { PF_EVAL = 0, PF_RHS, PF_FACTOR, PF_SOLVE, PF_STEP, PF_LINESEARCH, PF_UPDATE,
                 PF_ADMIT, PF_N };
static double g_prof_ms[PF_N];
static long long g_prof_rounds[PF_N];
static int g_prof_on = -1;
struct ProfClock {
  cudaStream_t st;
  int cur = -1;
  std::chrono::steady_clock::time_point t;
  explicit ProfClock(cudaStream_t s) : st(s) {
    if (g_prof_on < 0) {
      const char* e = std::getenv("COLLO_PROFILE");
      g_prof_on = (e && e[0] == '1') ? 1 : 0;
    }
    if (g_prof_on) t = std::chrono::steady_clock::now();
  }
  void mark(int next) {
    if (!g_prof_on) return;
    cudaStreamSynchronize(st);
    const auto now = std::chrono::steady_clock::now();
    if (cur >= 0) g_prof_ms[cur] += std::chrono::duration<double, std::milli>(now - t).count();
    t = now;
    cur = next;
  }
  void round(int ph) { if (g_prof_on) g_prof_rounds[ph]++; }
  ~ProfClock() { mark(-1); }
};

struct IpmInst {
  int slot = 0;
  collo_problem* prob = nullptr;
  Opt o;
  int status = RUNNING;
  double mu = 0.1, tau = 0.99, dw_last = 0.0, dw = 0.0, dc = 0.0;
  bool prev_reg = false;   // the last accepted factorization had dw > 0
  double theta_max = 0, theta_min = 0, err = INFINITY, phi = NAN;
  int acc = 0, it = 0, facs = 0, facs64 = 0, trials_total = 0, prec = 0, refine_total = 0;
  // MIXED path after a refinement failure: factor in FP64 until iteration
  // fp64_until, then try FP32 again; each further failure doubles the hold
  int fp64_until = 0, fp64_hold = 2;
  std::vector<std::pair<double, double>> filt;
  // line-search temporaries
  double theta_k = 0, phi_k = 0, gphi = 0, alpha = 0, alpha_min = 0, alpha_z = 0;
  bool ls_done = false, accepted = false, ftype = false;
  int trials = 0;
  std::chrono::steady_clock::time_point t0;
  double wall = 0;
};

// Initial point, forward sweep and the constraint norm at x0 for new instances.
// Initial parameters pushed into the bounds, bound duals 1, and the forward
// sweep of the states, for the instances of plan `which` (already set), on
// stream st.
static collo_status ipm_begin_sweep(Runner& R, int which, const Opt& o, cudaStream_t st) {
  const Plan& pl = R.plans[which];
  COLLO_CUDA(launch_init_point_b(R.d_insts, pl.act(), pl.A, o.kappa1, o.kappa2, st));
  COLLO_CUDA(launch_sweep_b(R.d_insts, pl.d_int + pl.off_sw_w, pl.n_sw_w, pl.smem_sw_w,
                            pl.d_int + pl.off_sw_c, pl.n_sw_c, pl.smem_sw_c, st));
  return COLLO_OK;
}

// The rest of an instance's start once its states are swept: lambda = 0, warm
// starts, the first evaluation and the barrier parameter.
static collo_status ipm_begin_rest(Runner& R, std::vector<IpmInst*>& ins);

static collo_status ipm_begin(Runner& R, std::vector<IpmInst*>& ins) {
  if (ins.empty()) return COLLO_OK;
  std::vector<int> slots;
  for (auto* I : ins) slots.push_back(I->slot);
  collo_status s = R.set_plan(3, slots);
  if (s != COLLO_OK) return s;
  if ((s = ipm_begin_sweep(R, 3, ins[0]->o, R.stream)) != COLLO_OK) return s;
  return ipm_begin_rest(R, ins);
}

static collo_status ipm_begin_rest(Runner& R, std::vector<IpmInst*>& ins) {
  if (ins.empty()) return COLLO_OK;
  std::vector<int> slots;
  for (auto* I : ins) slots.push_back(I->slot);
  collo_status s = R.set_plan(3, slots);
  if (s != COLLO_OK) return s;
  s = R.set_params(3, [&](int, int, InstParams& ip) { ip.alpha = 0.0; });
  if (s != COLLO_OK) return s;
  s = R.update(3, 2 /* lambda = 0 */);
  if (s != COLLO_OK) return s;
  // warm starts: the given states and multipliers replace the sweep's (theta
  // was pushed into its bounds from the start's values by the initial point)
  for (auto* I : ins) {
    collo_problem* pr = I->prob;
    if (!pr->has_start) continue;
    const size_t nz = (size_t)(pr->n_x - pr->P.p);
    COLLO_CUDA(cudaMemcpyAsync(pr->x, pr->start_x, nz * sizeof(double), cudaMemcpyDeviceToDevice,
                               R.stream));
    COLLO_CUDA(cudaMemcpyAsync(pr->lam, pr->start_lam, pr->n_c * sizeof(double),
                               cudaMemcpyDeviceToDevice, R.stream));
    pr->has_start = false;
  }
  s = R.eval(3, 1 /* V_X */, 0, 0, false);
  if (s != COLLO_OK) return s;
  s = R.read_outs();
  if (s != COLLO_OK) return s;
  for (auto* I : ins) {
    const double th = R.out(I->slot)[O_C1];
    I->theta_max = 1e4 * std::max(1.0, th);
    I->theta_min = 1e-4 * std::max(1.0, th);
    I->mu = I->o.mu_init;
    I->tau = std::max(I->o.tau_min, 1.0 - I->mu);
  }
  return COLLO_OK;
}

// One Newton iteration for every running instance in `ins`.
static collo_status ipm_iteration(Runner& R, std::vector<IpmInst*>& ins) {
  std::vector<IpmInst*> run;
  for (auto* I : ins)
    if (I->status == RUNNING) run.push_back(I);
  if (run.empty()) return COLLO_OK;
  std::map<int, IpmInst*> by_slot;
  std::vector<int> slots;
  for (auto* I : run) { slots.push_back(I->slot); by_slot[I->slot] = I; }
  auto fill_mu = [&](int, int s, InstParams& ip) {
    IpmInst* I = by_slot[s];
    ip.mu = I->mu; ip.tau = I->tau; ip.dw = I->dw; ip.dc = I->dc;
  };
  collo_status st;
  ProfClock prof(R.stream);
  prof.mark(PF_EVAL);
  // 1. derivatives and optimality measures
  if ((st = R.set_plan(0, slots)) != COLLO_OK) return st;
  if ((st = R.set_params(0, fill_mu)) != COLLO_OK) return st;
  if ((st = R.eval(0, 1 /* V_X */, 0, 2 /* V_LAM */, true)) != COLLO_OK) return st;
  {
    const Plan& pl = R.plans[0];
    COLLO_CUDA(launch_theta_prep_b(R.d_insts, pl.act(), pl.A, pl.d_prm, R.stream));
  }
  if ((st = R.resid(0, 0 /* R_DUAL */)) != COLLO_OK) return st;
  COLLO_CUDA(launch_vec_reduce_b(R.d_insts, R.plans[0].act(), R.plans[0].A, 0, R.stream));
  if ((st = R.read_outs()) != COLLO_OK) return st;
  std::vector<IpmInst*> cont;
  for (auto* I : run) {
    I->prob->evaluated = true;
    ++I->prob->eval_count;
    const double* o = R.out(I->slot);
    I->phi = o[O_PHI];
    const double cinf = o[O_CINF];
    if (!std::isfinite(I->phi) || !std::isfinite(o[O_C1])) { I->status = COLLO_ERR_NUMERIC; continue; }
    const int p = R.P(I->slot).p;
    const double nc = (double)R.h_insts[I->slot].n_c;
    const double wmax = o[O_WMAX], wmin = o[O_WMIN], zsum = o[O_ZSUM];
    const double dual = o[O_RX], lam1 = o[O_LAM1];
    const Opt& op = I->o;
    const double s_d = std::max(op.s_max, (lam1 + zsum) / (nc + 2 * p)) / op.s_max;
    const double s_c = std::max(op.s_max, zsum / (double)std::max(2 * p, 1)) / op.s_max;
    auto Emu = [&](double m) {
      double compl_ = p ? std::max(wmax - m, m - wmin) : 0.0;
      return std::max(std::max(dual / s_d, cinf), compl_ / s_c);
    };
    I->err = Emu(0.0);
    I->wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - I->t0).count();
    if (I->err <= op.tol) { I->status = COLLO_OK; continue; }
    I->acc = I->err <= op.acc_tol ? I->acc + 1 : 0;
    if (I->acc >= op.acc_iter) { I->status = COLLO_ACCEPTABLE; continue; }
    if (I->it >= op.max_iter) { I->status = COLLO_ERR_MAXITER; continue; }
    if (I->wall > op.max_wall) { I->status = COLLO_ERR_TIMEOUT; continue; }
    while (Emu(I->mu) <= op.kappa_eps * I->mu) {
      double nm = std::max(op.tol / 10.0, std::min(op.kappa_mu * I->mu, std::pow(I->mu, op.theta_mu)));
      if (nm >= I->mu) break;
      I->mu = nm;
      I->tau = std::max(op.tau_min, 1.0 - I->mu);
      I->filt.clear();
    }
    I->theta_k = o[O_C1] > 0 ? o[O_C1] : 0.0;
    I->prec = (op.precision == COLLO_PRECISION_MIXED && I->it >= I->fp64_until &&
               !(op.mixed_mu_switch > 0 && I->mu < op.mixed_mu_switch))
                  ? COLLO_PRECISION_MIXED : COLLO_PRECISION_FP64;
    I->dc = op.dc_coef * std::pow(I->mu, op.dc_exp);
    I->dw = 0.0;
    cont.push_back(I);
  }
  if (cont.empty()) return COLLO_OK;
  slots.clear();
  for (auto* I : cont) slots.push_back(I->slot);
  // 2. right-hand sides with the updated barrier parameters
  prof.mark(PF_RHS);
  if ((st = R.set_plan(0, slots)) != COLLO_OK) return st;
  if ((st = R.set_params(0, fill_mu)) != COLLO_OK) return st;
  {
    const Plan& pl = R.plans[0];
    COLLO_CUDA(launch_theta_prep_b(R.d_insts, pl.act(), pl.A, pl.d_prm, R.stream));
  }
  if ((st = R.resid(0, 1 /* R_RHS */)) != COLLO_OK) return st;
  // 3. factorization with inertia correction (per precision group), then
  // 4. solve with FP64 refinement.  An instance of the MIXED path whose
  // refinement fails (relative residual above ESCALATE_REL after refine_max
  // sweeps, or stalled above it) is factored and solved again in FP64, and
  // factors in FP64 for the next 2, 4, 8, ... iterations (doubling after each
  // failure) before trying FP32 again.
  std::vector<IpmInst*> go;
  auto factor_solve = [&](std::vector<IpmInst*> fac, std::vector<IpmInst*>& redo) -> collo_status {
    std::vector<IpmInst*> list = fac;
    prof.mark(PF_FACTOR);
    // Inertia correction (Wachter & Biegler 2006, Section 3.1): the candidate
    // regularisations of one iteration are 0, then c1 = 1e-4 or
    // max(dw_min, dw_last / 3), then c1 times 100 (no history) or 8, ... until
    // the inertia is right.  From the second round on, each instance factors two
    // consecutive candidates at once (the second in its shadow slot) and takes
    // the first of the two, in sequence order, whose inertia is right: the same
    // regularisation as the one-at-a-time sequence, in fewer rounds.  An
    // instance whose last accepted factorization needed dw > 0 is likely to
    // need it again, so it pairs 0 with its first candidate from the first
    // round on.
    std::map<int, double> dw2;   // slot -> second candidate of this round (0: none)
    for (auto* I : fac) {
      if (!I->prev_reg || I->dw != 0.0 || I->dw_last == 0.0) continue;
      const double c1 = std::max(I->o.dw_min, I->o.kw_minus * I->dw_last);
      if (c1 <= I->o.dw_max) dw2[I->slot] = c1;
    }
    while (!fac.empty()) {
      prof.round(PF_FACTOR);
      std::vector<int> gr[2];
      for (auto* I : fac) {
        const int g = I->prec == COLLO_PRECISION_MIXED ? 1 : 0;
        gr[g].push_back(I->slot);
        auto it = dw2.find(I->slot);
        if (it != dw2.end() && it->second > 0) gr[g].push_back(R.shadow(I->slot));
      }
      for (int g = 0; g < 2; ++g) {
        if (gr[g].empty()) continue;
        const int pl = g == 1 ? 1 : 2;
        if ((st = R.set_plan(pl, gr[g])) != COLLO_OK) return st;
        if ((st = R.set_params(pl, [&](int k, int s, InstParams& ip) {
               if (s >= R.capacity) {
                 fill_mu(k, s - R.capacity, ip);
                 ip.dw = dw2[s - R.capacity];
               } else {
                 fill_mu(k, s, ip);
               }
             })) != COLLO_OK)
          return st;
        if ((st = R.factor(pl, g ? COLLO_PRECISION_MIXED : COLLO_PRECISION_FP64)) != COLLO_OK)
          return st;
      }
      if ((st = R.read_outs()) != COLLO_OK) return st;
      if ((st = R.check_barrier()) != COLLO_OK) return st;
      auto inertia_ok = [&](int s, int base) {
        long long in[3];
        std::memcpy(in, R.out(s) + O_INERT, sizeof(in));
        return in[0] == R.h_insts[base].n_x && in[1] == R.h_insts[base].n_c && in[2] == 0;
      };
      std::vector<IpmInst*> again;
      for (auto* I : fac) {
        const double second = dw2.count(I->slot) ? dw2[I->slot] : 0.0;
        const int nf = second > 0 ? 2 : 1;
        I->facs += nf;
        if (I->prec != COLLO_PRECISION_MIXED) I->facs64 += nf;
        bool good = inertia_ok(I->slot, I->slot);
        if (!good && second > 0 && inertia_ok(R.shadow(I->slot), I->slot)) {
          swap_spare(I->prob, I->prec);
          if ((st = R.attach(I->slot, I->prob)) != COLLO_OK) return st;
          I->dw = second;
          good = true;
        }
        if (good) {
          I->prob->factored = I->prec;
          I->prob->fac_dw = I->dw;
          I->prob->fac_dc = I->dc;
          if (I->dw > 0) I->dw_last = I->dw;
          I->prev_reg = I->dw > 0;
          dw2.erase(I->slot);
          continue;
        }
        const Opt& op = I->o;
        const double last = second > 0 ? second : I->dw;
        const double mult = I->dw_last == 0.0 ? op.kw_plus_bar : op.kw_plus;
        const double c1 = last == 0.0 ? (I->dw_last == 0.0 ? op.dw_0
                                                          : std::max(op.dw_min, op.kw_minus * I->dw_last))
                                      : last * mult;
        if (c1 > op.dw_max) { I->status = COLLO_ERR_INERTIA; dw2.erase(I->slot); continue; }
        I->dw = c1;
        dw2[I->slot] = c1 * mult <= op.dw_max ? c1 * mult : 0.0;
        again.push_back(I);
      }
      fac = again;
    }
    std::vector<IpmInst*> run_now;
    for (auto* I : list)
      if (I->status == RUNNING) run_now.push_back(I);
    if (run_now.empty()) return COLLO_OK;
    std::vector<int> sl;
    for (auto* I : run_now) sl.push_back(I->slot);
    prof.mark(PF_SOLVE);
    if ((st = R.set_plan(0, sl)) != COLLO_OK) return st;
    std::vector<int> prec_of_slot(R.capacity, 0);
    std::vector<double> dwv, dcv;
    for (auto* I : run_now) { prec_of_slot[I->slot] = I->prec; dwv.push_back(I->dw); dcv.push_back(I->dc); }
    std::vector<int> sweeps;
    std::vector<double> rel;
    const Opt& op = run_now[0]->o;
    if ((st = solve_refine(R, 0, prec_of_slot, dwv, dcv, op.refine_max, op.refine_tol, sweeps, rel)) != COLLO_OK)
      return st;
    int max_sw = 0;
    for (int v : sweeps) max_sw = std::max(max_sw, v);
    for (int k = 0; k <= max_sw; ++k) prof.round(PF_SOLVE);
    for (size_t k = 0; k < run_now.size(); ++k) {
      IpmInst* I = run_now[k];
      I->refine_total += sweeps[k];
      if (I->prec == COLLO_PRECISION_MIXED && !(rel[k] <= ESCALATE_REL)) {
        I->fp64_until = I->it + I->fp64_hold;
        I->fp64_hold *= 2;
        I->prec = COLLO_PRECISION_FP64;
        I->dw = 0.0;
        redo.push_back(I);
        continue;
      }
      if (!std::isfinite(rel[k])) I->status = COLLO_ERR_NUMERIC;
    }
    return COLLO_OK;
  };
  {
    std::vector<IpmInst*> redo, none;
    if ((st = factor_solve(cont, redo)) != COLLO_OK) return st;
    if (!redo.empty() && (st = factor_solve(redo, none)) != COLLO_OK) return st;
  }
  for (auto* I : cont)
    if (I->status == RUNNING) go.push_back(I);
  if (go.empty()) return COLLO_OK;
  slots.clear();
  for (auto* I : go) slots.push_back(I->slot);
  // 5. step sizes
  prof.mark(PF_STEP);
  if ((st = R.set_plan(0, slots)) != COLLO_OK) return st;
  if ((st = R.set_params(0, fill_mu)) != COLLO_OK) return st;
  {
    const Plan& pl = R.plans[0];
    COLLO_CUDA(launch_theta_step_b(R.d_insts, pl.act(), pl.A, pl.d_prm, R.stream));
    COLLO_CUDA(launch_vec_reduce_b(R.d_insts, pl.act(), pl.A, 1, R.stream));
  }
  if ((st = R.read_outs()) != COLLO_OK) return st;
  std::vector<IpmInst*> ls;
  for (auto* I : go) {
    if (I->status != RUNNING) continue;
    const double* o = R.out(I->slot);
    const Opt& op = I->o;
    const double alpha_max = o[O_AMAX];
    I->alpha_z = o[O_AZ];
    I->gphi = o[O_GDX] + o[O_GPHI];
    I->phi_k = I->phi - I->mu * o[O_LOG];
    const double tk = I->theta_k, g = I->gphi;
    if (g < 0) {
      if (tk <= I->theta_min)
        I->alpha_min = op.gamma_alpha * std::min(std::min(op.gamma_theta, op.gamma_phi * tk / (-g)),
                                                 op.delta * std::pow(tk, op.s_theta) / std::pow(-g, op.s_phi));
      else
        I->alpha_min = op.gamma_alpha * std::min(op.gamma_theta, op.gamma_phi * tk / (-g));
    } else {
      I->alpha_min = op.gamma_alpha * op.gamma_theta;
    }
    I->alpha = alpha_max;
    I->accepted = false;
    I->trials = 0;
    ls.push_back(I);
  }
  // 6. backtracking filter line search, all instances in step.  From the second
  // round on, an instance still backtracking evaluates its next two trial steps
  // (alpha and alpha / 2, the second in its shadow slot) in the same round and
  // takes the first of them, in sequence order, that is acceptable: the same
  // step, the same trial count, in fewer rounds.
  std::vector<IpmInst*> trying;
  for (auto* I : ls) {
    if (I->alpha >= I->alpha_min) trying.push_back(I);
    else I->status = COLLO_ERR_LINESEARCH;
  }
  // trial point acceptance (filter, switching condition, Armijo / sufficient
  // progress) of the trial at I->alpha whose evaluation is in out slot o
  auto acceptable = [&](IpmInst* I, const double* o) {
    const Opt& op = I->o;
    const double phit = o[O_PHI], thetat = o[O_C1];
    if (!(std::isfinite(phit) && std::isfinite(thetat) && o[O_TOK] > 0.5)) return false;
    const double phibt = phit - I->mu * o[O_TLOG];
    bool ok = std::isfinite(phibt) && thetat < I->theta_max;
    if (ok)
      for (auto& f : I->filt)
        if (thetat >= f.first && phibt >= f.second) { ok = false; break; }
    if (!ok) return false;
    const bool sw = I->gphi < 0 &&
                    I->alpha * std::pow(-I->gphi, op.s_phi) > op.delta * std::pow(I->theta_k, op.s_theta);
    if (I->theta_k <= I->theta_min && sw) {
      I->ftype = true;
      return phibt <= I->phi_k + op.eta_phi * I->alpha * I->gphi;
    }
    I->ftype = false;
    return thetat <= (1.0 - op.gamma_theta) * I->theta_k || phibt <= I->phi_k - op.gamma_phi * I->theta_k;
  };
  prof.mark(PF_LINESEARCH);
  for (int round = 0; !trying.empty(); ++round) {
    prof.round(PF_LINESEARCH);
    slots.clear();
    std::map<int, double> half;   // slot -> second trial step of this round
    for (auto* I : trying) {
      slots.push_back(I->slot);
      if (round > 0 && 0.5 * I->alpha >= I->alpha_min) {
        half[I->slot] = 0.5 * I->alpha;
        slots.push_back(R.shadow(I->slot));
      }
    }
    if ((st = R.set_plan(1, slots)) != COLLO_OK) return st;
    if ((st = R.set_params(1, [&](int, int s, InstParams& ip) {
           ip.alpha = s >= R.capacity ? half[s - R.capacity] : by_slot[s]->alpha;
         })) != COLLO_OK)
      return st;
    if ((st = R.eval(1, 1 /* V_X */, 5 /* V_KB */, 0, false)) != COLLO_OK) return st;
    {
      const Plan& pl = R.plans[1];
      COLLO_CUDA(launch_trial_barrier_b(R.d_insts, pl.act(), pl.A, pl.d_prm, R.stream));
    }
    if ((st = R.read_outs()) != COLLO_OK) return st;
    std::vector<IpmInst*> next;
    for (auto* I : trying) {
      I->trials++;
      if (acceptable(I, R.out(I->slot))) { I->accepted = true; continue; }
      I->alpha *= 0.5;
      if (I->alpha < I->alpha_min) { I->status = COLLO_ERR_LINESEARCH; continue; }
      if (half.count(I->slot)) {
        I->trials++;
        if (acceptable(I, R.out(R.shadow(I->slot)))) { I->accepted = true; continue; }
        I->alpha *= 0.5;
        if (I->alpha < I->alpha_min) { I->status = COLLO_ERR_LINESEARCH; continue; }
      }
      next.push_back(I);
    }
    trying = next;
  }
  // 7. accept the steps
  prof.mark(PF_UPDATE);
  std::vector<IpmInst*> upd;
  for (auto* I : ls) {
    I->trials_total += I->trials;
    if (!I->accepted) continue;
    const Opt& op = I->o;
    if (!I->ftype) I->filt.push_back({(1.0 - op.gamma_theta) * I->theta_k, I->phi_k - op.gamma_phi * I->theta_k});
    upd.push_back(I);
  }
  if (!upd.empty()) {
    slots.clear();
    for (auto* I : upd) slots.push_back(I->slot);
    if ((st = R.set_plan(0, slots)) != COLLO_OK) return st;
    if ((st = R.set_params(0, [&](int, int s, InstParams& ip) {
           IpmInst* I = by_slot[s];
           ip.alpha = I->alpha; ip.alpha_z = I->alpha_z; ip.mu = I->mu; ip.ksig = I->o.kappa_sigma;
         })) != COLLO_OK)
      return st;
    if ((st = R.update(0, 0)) != COLLO_OK) return st;
    for (auto* I : upd) {
      if (I->o.verbose)
        std::printf("[%d] iter %4d phi %.10e err %.3e mu %.3e dw %.2e alpha %.3e ls %d %s\n",
                    I->slot, I->it, I->phi, I->err, I->mu, I->dw, I->alpha, I->trials,
                    I->prec == COLLO_PRECISION_MIXED ? "fp32+ir" : "fp64");
      I->it++;
    }
  }
  return COLLO_OK;
}

static collo_status ipm_finish(Runner& R, IpmInst& I, collo_result* res) {
  collo_problem* pr = I.prob;
  cudaStream_t st = R.stream;
  const int p = pr->P.p;
  const size_t nx = pr->n_x, nc = pr->n_c, nz = nx - p;
  res->status = I.status;
  res->iterations = I.it;
  res->factorizations = I.facs;
  res->line_search_trials = I.trials_total;
  res->refinement_sweeps = I.refine_total;
  res->fp64_factorizations = I.facs64;
  res->phi = I.phi;
  res->kkt_error = I.err;
  res->mu = I.mu;
  if (res->theta && p)
    COLLO_CUDA(cudaMemcpyAsync(res->theta, pr->x + nz, p * sizeof(double), cudaMemcpyDefault, st));
  if (res->x) COLLO_CUDA(cudaMemcpyAsync(res->x, pr->x, nx * sizeof(double), cudaMemcpyDefault, st));
  if (res->lambda)
    COLLO_CUDA(cudaMemcpyAsync(res->lambda, pr->lam, nc * sizeof(double), cudaMemcpyDefault, st));
  COLLO_CUDA(cudaStreamSynchronize(st));
  res->wall_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - I.t0).count();
  return COLLO_OK;
}

static collo_status ipm_prepare(Runner& R, int slot, collo_problem* pr, const double* theta0,
                                const Opt& o, IpmInst& I) {
  collo_status s = ensure_factor_storage(pr, COLLO_PRECISION_FP64);
  if (s != COLLO_OK) return s;
  if ((s = ensure_spare_storage(pr, COLLO_PRECISION_FP64)) != COLLO_OK) return s;
  if (o.precision == COLLO_PRECISION_MIXED) {
    if ((s = ensure_factor_storage(pr, COLLO_PRECISION_MIXED)) != COLLO_OK) return s;
    if ((s = ensure_spare_storage(pr, COLLO_PRECISION_MIXED)) != COLLO_OK) return s;
  }
  if ((s = R.attach(slot, pr)) != COLLO_OK) return s;
  // a warm start (collo_problem_set_start) supplies theta0 from its x
  const double* th = pr->has_start ? pr->start_x + (pr->n_x - pr->P.p) : theta0;
  if (pr->P.p)
    COLLO_CUDA(cudaMemcpyAsync(pr->inst.th0, th, pr->P.p * sizeof(double), cudaMemcpyDefault,
                               R.stream));
  I = IpmInst();
  I.slot = slot;
  I.prob = pr;
  I.o = o;
  I.t0 = std::chrono::steady_clock::now();
  return COLLO_OK;
}

// ---- single-instance operations through the problem's own runner -------------------
collo_status runner_eval(collo_problem* pr, double obj_factor) {
  Runner* R = nullptr;
  collo_status s = self_attach(pr, &R);
  if (s != COLLO_OK) return s;
  if ((s = R->set_plan(0, {0})) != COLLO_OK) return s;
  if ((s = R->set_params(0, [&](int, int, InstParams& ip) { ip.obj_factor = obj_factor; })) != COLLO_OK)
    return s;
  return R->eval(0, 3 /* V_STAGE_X */, 0, 4 /* V_STAGE_L */, true);
}

collo_status runner_factor(collo_problem* pr, int prec, double dw, double dc, long long inertia[3]) {
  collo_status s = ensure_factor_storage(pr, prec);
  if (s != COLLO_OK) return s;
  Runner* R = nullptr;
  if ((s = self_attach(pr, &R)) != COLLO_OK) return s;
  if ((s = R->set_plan(0, {0})) != COLLO_OK) return s;
  if ((s = R->set_params(0, [&](int, int, InstParams& ip) { ip.dw = dw; ip.dc = dc; })) != COLLO_OK)
    return s;
  if ((s = R->factor(0, prec)) != COLLO_OK) return s;
  if ((s = R->read_outs()) != COLLO_OK) return s;
  if ((s = R->check_barrier()) != COLLO_OK) return s;
  std::memcpy(inertia, R->out(0) + O_INERT, 3 * sizeof(long long));
  pr->factored = prec;
  pr->fac_dw = dw;
  pr->fac_dc = dc;
  return COLLO_OK;
}

// Solve with the right-hand side in ka into kb (refined in FP64).
collo_status runner_solve(collo_problem* pr, int refine_max, double refine_tol, int* sweeps,
                          double* resid) {
  Runner* R = nullptr;
  collo_status s = self_runner(pr, &R);
  if (s != COLLO_OK) return s;
  if ((s = R->set_plan(0, {0})) != COLLO_OK) return s;
  std::vector<int> prec_of_slot{pr->factored};
  std::vector<double> dw{pr->fac_dw}, dc{pr->fac_dc};
  std::vector<int> sw;
  std::vector<double> rel;
  if ((s = solve_refine(*R, 0, prec_of_slot, dw, dc, refine_max, refine_tol, sw, rel)) != COLLO_OK)
    return s;
  if (sweeps) *sweeps = sw[0];
  if (resid) *resid = rel[0];
  if (!std::isfinite(rel[0])) { set_error("non-finite KKT solution"); return COLLO_ERR_NUMERIC; }
  return COLLO_OK;
}

// CUDA-event timing of one batched phase of this problem (batch of one):
// 1 factorization, 2 solve (no refinement), 3 evaluation with derivatives.
collo_status runner_time_phase(collo_problem* pr, int phase, int prec, int reps, double* ms) {
  collo_status s = ensure_factor_storage(pr, prec);
  if (s != COLLO_OK) return s;
  Runner* R = nullptr;
  if ((s = self_attach(pr, &R)) != COLLO_OK) return s;
  if ((s = R->set_plan(0, {0})) != COLLO_OK) return s;
  if ((s = R->set_params(0, [&](int, int, InstParams& ip) { ip.dw = pr->fac_dw; ip.dc = pr->fac_dc; })) != COLLO_OK)
    return s;
  auto run = [&]() -> collo_status {
    if (phase == 1) return R->factor(0, prec);
    if (phase == 2) return R->solve(0, prec, 0);
    return R->eval(0, 1 /* V_X */, 0, 2 /* V_LAM */, true);
  };
  if ((s = run()) != COLLO_OK) return s;
  cudaEvent_t e0, e1;
  COLLO_CUDA(cudaEventCreate(&e0));
  COLLO_CUDA(cudaEventCreate(&e1));
  COLLO_CUDA(cudaEventRecord(e0, R->stream));
  for (int k = 0; k < reps; ++k)
    if ((s = run()) != COLLO_OK) return s;
  COLLO_CUDA(cudaEventRecord(e1, R->stream));
  COLLO_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / reps;
  if (phase == 1) pr->factored = prec;
  return R->check_barrier();
}

}  // namespace collo

using namespace collo;

// ---- continuous-batching server --------------------------------------------------------
struct collo_server {
  Runner R;
  Opt o;
  int64_t budget = 0;
  int64_t active_bytes = 0;   // held by admitted jobs' problems
  int64_t peak_bytes = 0;     // largest active_bytes so far
  long long newton_steps = 0; // Newton steps taken by all jobs
  long long finished = 0;     // jobs with a final status
  long long converged = 0;    // ... of them solved (COLLO_OK or COLLO_ACCEPTABLE)
  long long next_ticket = 1;
  struct Job {
    long long ticket;
    collo_problem* prob;
    std::vector<double> theta0;
    IpmInst I;
    int slot = -1;
    bool done = false;
    int64_t bytes = 0;   // device bytes its problem holds while admitted
    collo_result res{};
  };
  std::deque<Job*> waiting;
  std::vector<Job*> slots;            // slot -> job (null: free)
  int admit_min = 1;                  // admit when this many slots are free (or none is busy)
  std::map<long long, Job*> jobs;
  std::mutex mu;
  // Admitted jobs whose forward sweeps run on the side stream while the
  // other jobs keep stepping; they join the Newton steps once side_ev has
  // completed.  One such group at a time (it owns plan 4).
  cudaStream_t side = nullptr;
  cudaEvent_t side_ev = nullptr;      // end of the group's sweeps
  cudaEvent_t main_ev = nullptr;      // the group's set-up on the main stream
  std::vector<Job*> sweeping;
  ~collo_server() {
    if (side) { cudaStreamSynchronize(side); cudaStreamDestroy(side); }
    if (side_ev) cudaEventDestroy(side_ev);
    if (main_ev) cudaEventDestroy(main_ev);
    for (auto& kv : jobs) delete kv.second;
  }
};

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
  o->mixed_mu_switch = 0.0;
  o->refine_max = 10;
  o->refine_tol = 1e-10;
  o->verbose = 0;
}

collo_status collo_initial_states(collo_problem* prob, const double* theta, double* x_out,
                                  int* failures) {
  if (!prob || !theta) { set_error("NULL argument"); return COLLO_ERR_INVALID_ARG; }
  COLLO_CUDA(cudaSetDevice(prob->device));
  Runner* R = nullptr;
  collo_status s = self_attach(prob, &R);
  if (s != COLLO_OK) return s;
  const size_t nz = (size_t)prob->P.N * prob->P.np * prob->P.n;
  if (prob->P.p)
    COLLO_CUDA(cudaMemcpyAsync(prob->x + nz, theta, prob->P.p * sizeof(double), cudaMemcpyDefault,
                               R->stream));
  if ((s = R->set_plan(3, {0})) != COLLO_OK) return s;
  const Plan& pl = R->plans[3];
  COLLO_CUDA(launch_sweep_b(R->d_insts, pl.d_int + pl.off_sw_w, pl.n_sw_w, pl.smem_sw_w,
                            pl.d_int + pl.off_sw_c, pl.n_sw_c, pl.smem_sw_c, R->stream));
  int f = 0;
  COLLO_CUDA(cudaMemcpyAsync(&f, prob->fails, sizeof(int), cudaMemcpyDeviceToHost, R->stream));
  if (x_out)
    COLLO_CUDA(cudaMemcpyAsync(x_out, prob->x, prob->n_x * sizeof(double), cudaMemcpyDefault, R->stream));
  COLLO_CUDA(cudaStreamSynchronize(R->stream));
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
  Runner* R = nullptr;
  collo_status s = self_runner(prob, &R);
  if (s != COLLO_OK) return s;
  Opt o = make_opt(opts);
  IpmInst I;
  if ((s = ipm_prepare(*R, 0, prob, theta0, o, I)) != COLLO_OK) return s;
  std::vector<IpmInst*> ins{&I};
  if ((s = ipm_begin(*R, ins)) != COLLO_OK) return res->status = s;
  while (I.status == RUNNING) {
    s = ipm_iteration(*R, ins);
    if (s != COLLO_OK) { I.status = s; break; }
  }
  s = ipm_finish(*R, I, res);
  if (s != COLLO_OK) return s;
  return res->status;
}

// ---- batches -------------------------------------------------------------------------
struct collo_batch_impl;

collo_status collo_batch_solve(collo_problem* const* probs, int count, const double* const* theta0,
                               const collo_ipm_options* opts, collo_result* results) {
  if (!probs || count < 1 || !theta0 || !results) {
    set_error("bad argument");
    return COLLO_ERR_INVALID_ARG;
  }
  const int dev = probs[0]->device;
  for (int i = 0; i < count; ++i)
    if (!probs[i] || probs[i]->device != dev || (probs[i]->P.p > 0 && !theta0[i])) {
      set_error("batch members must be valid problems of one device with theta0");
      return COLLO_ERR_INVALID_ARG;
    }
  COLLO_CUDA(cudaSetDevice(dev));
  Runner R;
  collo_status s = R.init(count, dev, probs[0]->stream);   // runs on the first problem's stream
  if (s != COLLO_OK) return s;
  Opt o = make_opt(opts);
  std::vector<IpmInst> I(count);
  std::vector<IpmInst*> ins;
  for (int i = 0; i < count; ++i) {
    if ((s = ipm_prepare(R, i, probs[i], theta0[i], o, I[i])) != COLLO_OK) return s;
    ins.push_back(&I[i]);
  }
  if ((s = ipm_begin(R, ins)) != COLLO_OK) return s;
  for (;;) {
    bool any = false;
    for (auto* p : ins) any = any || p->status == RUNNING;
    if (!any) break;
    s = ipm_iteration(R, ins);
    if (s != COLLO_OK) {
      for (auto* p : ins) if (p->status == RUNNING) p->status = s;
      break;
    }
  }
  for (int i = 0; i < count; ++i)
    if ((s = ipm_finish(R, I[i], &results[i])) != COLLO_OK) return s;
  return COLLO_OK;
}

// CUDA-event timing of one batched phase over problems that each hold an
// evaluated iterate and a factorization (e.g. after collo_batch_solve):
// phase 1 factorization, 2 solve (no refinement), 3 evaluation.
collo_status collo_batch_time_phase(collo_problem* const* probs, int count, int phase,
                                    int precision, int reps, double* ms_per_launch) {
  if (!probs || count < 1 || reps < 1 || !ms_per_launch || phase < 1 || phase > 7) {
    set_error("bad argument");
    return COLLO_ERR_INVALID_ARG;
  }
  const int dev = probs[0]->device;
  COLLO_CUDA(cudaSetDevice(dev));
  Runner R;
  collo_status s = R.init(count, dev, nullptr);
  if (s != COLLO_OK) return s;
  std::vector<int> slots;
  for (int i = 0; i < count; ++i) {
    if (!probs[i]->evaluated) { set_error("problem not evaluated"); return COLLO_ERR_NOT_EVALUATED; }
    if ((s = ensure_factor_storage(probs[i], precision)) != COLLO_OK) return s;
    if ((s = R.attach(i, probs[i])) != COLLO_OK) return s;
    slots.push_back(i);
  }
  if ((s = R.set_plan(0, slots)) != COLLO_OK) return s;
  if ((s = R.set_params(0, [&](int, int sl, InstParams& ip) {
         ip.dw = probs[sl]->fac_dw; ip.dc = probs[sl]->fac_dc; })) != COLLO_OK)
    return s;
  auto run = [&]() -> collo_status {
    if (phase == 1) return R.factor(0, precision);
    if (phase == 2) return R.solve(0, precision, 0);
    if (phase == 4) return R.factor(0, precision, 1 | 4);
    if (phase == 5) return R.factor(0, precision, 2);
    if (phase == 6) return R.factor(0, precision, 4);
    if (phase == 7) return R.factor(0, precision, 1);
    return R.eval(0, 1, 0, 2, true);
  };
  if ((phase == 2 || phase == 5) && (s = R.factor(0, precision)) != COLLO_OK) return s;
  if ((phase == 6 || phase == 7) && (s = R.factor(0, precision)) != COLLO_OK) return s;
  if ((s = run()) != COLLO_OK) return s;
  cudaEvent_t e0, e1;
  COLLO_CUDA(cudaEventCreate(&e0));
  COLLO_CUDA(cudaEventCreate(&e1));
  COLLO_CUDA(cudaEventRecord(e0, R.stream));
  for (int k = 0; k < reps; ++k)
    if ((s = run()) != COLLO_OK) return s;
  COLLO_CUDA(cudaEventRecord(e1, R.stream));
  COLLO_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_per_launch = t / reps;
  for (int i = 0; i < count; ++i)
    if (phase <= 2 || phase >= 5) probs[i]->factored = precision;
  return R.check_barrier();
}

// ---- server --------------------------------------------------------------------------
collo_status collo_server_create(int max_slots, int64_t budget_bytes, const collo_ipm_options* opts,
                                 int device, collo_server** out) {
  if (!out || max_slots < 1) { set_error("bad argument"); return COLLO_ERR_INVALID_ARG; }
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaSetDevice failed");
    return COLLO_ERR_DEVICE;
  }
  std::unique_ptr<collo_server> sv(new collo_server());
  collo_status s = sv->R.init(max_slots, device, nullptr);
  if (s != COLLO_OK) return s;
  COLLO_CUDA(cudaStreamCreateWithFlags(&sv->side, cudaStreamNonBlocking));
  COLLO_CUDA(cudaEventCreateWithFlags(&sv->side_ev, cudaEventDisableTiming));
  COLLO_CUDA(cudaEventCreateWithFlags(&sv->main_ev, cudaEventDisableTiming));
  sv->o = make_opt(opts);
  sv->budget = budget_bytes;
  sv->slots.assign(max_slots, nullptr);
  // factorization stores come from the device's default stream-ordered pool;
  // let it keep up to the budget (64 GiB without one) of freed memory for the
  // next admissions instead of returning it at every synchronisation
  {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t keep = 0;
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      const uint64_t want = budget_bytes > 0 ? (uint64_t)budget_bytes : (uint64_t)64 << 30;
      if (want > keep) cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, (void*)&want);
    }
    cudaGetLastError();
  }
  *out = sv.release();
  return COLLO_OK;
}

collo_status collo_server_submit(collo_server* sv, collo_problem* prob, const double* theta0,
                                 long long* ticket) {
  if (!sv || !prob || !ticket || (prob->P.p > 0 && !theta0)) {
    set_error("bad argument");
    return COLLO_ERR_INVALID_ARG;
  }
  auto* j = new collo_server::Job();
  j->ticket = sv->next_ticket++;
  j->prob = prob;
  j->theta0.assign(theta0, theta0 + prob->P.p);
  sv->jobs[j->ticket] = j;
  sv->waiting.push_back(j);
  *ticket = j->ticket;
  return COLLO_OK;
}

collo_status collo_server_step(collo_server* sv, int* n_active, int* n_waiting) {
  if (!sv) { set_error("NULL server"); return COLLO_ERR_INVALID_ARG; }
  COLLO_CUDA(cudaSetDevice(sv->R.device));
  Runner& R = sv->R;
  collo_status s;
  // Jobs whose forward sweeps (side stream) have finished join the Newton
  // steps: their start is completed on the main stream after the sweeps.
  std::vector<IpmInst*> fresh;
  if (!sv->sweeping.empty()) {
    const cudaError_t q = cudaEventQuery(sv->side_ev);
    if (q != cudaSuccess && q != cudaErrorNotReady) COLLO_CUDA(q);
    if (q == cudaSuccess) {
      COLLO_CUDA(cudaStreamWaitEvent(R.stream, sv->side_ev, 0));
      for (auto* j : sv->sweeping) fresh.push_back(&j->I);
      sv->sweeping.clear();
      R.reserve_sms = 0;
    }
  }
  // admit waiting jobs into free slots within the device-memory budget, in
  // groups of at least admit_min (a group's forward sweeps run one block per
  // job on the side stream, beside the other jobs' Newton steps, whose
  // cooperative grids leave that many SMs free meanwhile; one group at a
  // time).  A job's footprint is its problem's arrays plus every
  // factorization store the solve allocates (counted before they exist); the
  // stores are allocated at admission and freed when the job retires.  Jobs
  // are admitted in submission order; one larger than the whole budget fails
  // with OOM.
  std::vector<collo_server::Job*> group;
  int n_free = 0, n_busy = 0;
  for (auto* j : sv->slots) (j ? n_busy : n_free)++;
  const bool admit = sv->sweeping.empty() &&
                     (n_busy == 0 || n_free >= std::min(sv->admit_min, (int)sv->slots.size()));
  while (admit && !sv->waiting.empty()) {
    auto* j = sv->waiting.front();
    int slot = -1;
    for (int k = 0; k < (int)sv->slots.size(); ++k)
      if (!sv->slots[k]) { slot = k; break; }
    if (slot < 0) break;
    const int64_t need = problem_solve_bytes(j->prob, sv->o.precision);
    if (sv->budget > 0 && need > sv->budget) {
      sv->waiting.pop_front();
      j->res = collo_result{};
      j->res.status = COLLO_ERR_OOM;
      j->done = true;
      sv->finished++;
      continue;
    }
    if (sv->budget > 0 && sv->active_bytes + need > sv->budget) break;
    sv->waiting.pop_front();
    if ((s = ipm_prepare(R, slot, j->prob, j->theta0.data(), sv->o, j->I)) != COLLO_OK) return s;
    j->slot = slot;
    j->bytes = problem_held_bytes(j->prob);
    sv->slots[slot] = j;
    sv->active_bytes += j->bytes;
    sv->peak_bytes = std::max(sv->peak_bytes, sv->active_bytes);
    group.push_back(j);
  }
  if (!group.empty()) {
    ProfClock prof(R.stream);
    prof.mark(PF_ADMIT);
    prof.round(PF_ADMIT);
    std::vector<int> gs;
    for (auto* j : group) gs.push_back(j->slot);
    if ((s = R.set_plan(4, gs)) != COLLO_OK) return s;
    if (n_busy == 0) {
      // nothing else to run: sweep on the main stream and start at once
      if ((s = ipm_begin_sweep(R, 4, sv->o, R.stream)) != COLLO_OK) return s;
      for (auto* j : group) fresh.push_back(&j->I);
    } else {
      // the plan upload and the jobs' set-up precede the sweeps
      COLLO_CUDA(cudaEventRecord(sv->main_ev, R.stream));
      COLLO_CUDA(cudaStreamWaitEvent(sv->side, sv->main_ev, 0));
      if ((s = ipm_begin_sweep(R, 4, sv->o, sv->side)) != COLLO_OK) return s;
      COLLO_CUDA(cudaEventRecord(sv->side_ev, sv->side));
      sv->sweeping = group;
      R.reserve_sms = (int)group.size();   // one block per job's sweep
    }
  }
  {
    ProfClock prof(R.stream);
    if (!fresh.empty()) { prof.mark(PF_ADMIT); }
    if ((s = ipm_begin_rest(R, fresh)) != COLLO_OK) return s;
  }
  std::vector<IpmInst*> act;
  long long its0 = 0, its1 = 0;
  for (auto* j : sv->slots) {
    if (!j) continue;
    bool sweeping = false;
    for (auto* w : sv->sweeping) sweeping = sweeping || w == j;
    if (!sweeping) { act.push_back(&j->I); its0 += j->I.it; }
  }
  if ((s = ipm_iteration(R, act)) != COLLO_OK) return s;
  for (auto* I : act) its1 += I->it;
  sv->newton_steps += its1 - its0;
  // retire finished jobs
  for (int k = 0; k < (int)sv->slots.size(); ++k) {
    auto* j = sv->slots[k];
    if (!j || j->I.status == RUNNING) continue;
    j->res = collo_result{};
    if ((s = ipm_finish(R, j->I, &j->res)) != COLLO_OK) return s;
    j->done = true;
    sv->finished++;
    if (j->res.status == COLLO_OK || j->res.status == COLLO_ACCEPTABLE) sv->converged++;
    // its factorization stores go back in stream order after its last kernels
    release_factor_storage(j->prob, R.stream);
    sv->active_bytes -= j->bytes;
    sv->slots[k] = nullptr;
  }
  int a = 0;
  for (auto* j : sv->slots) a += j ? 1 : 0;
  if (n_active) *n_active = a;
  if (n_waiting) *n_waiting = (int)sv->waiting.size();
  return COLLO_OK;
}

int collo_phase_profile(double* ms, long long* rounds, int n, int reset) {
  const int m = std::min(n, (int)PF_N);
  for (int k = 0; k < m; ++k) {
    if (ms) ms[k] = g_prof_ms[k];
    if (rounds) rounds[k] = g_prof_rounds[k];
  }
  if (reset)
    for (int k = 0; k < PF_N; ++k) { g_prof_ms[k] = 0.0; g_prof_rounds[k] = 0; }
  return g_prof_on > 0 ? (int)PF_N : 0;
}

collo_status collo_server_memory(collo_server* sv, int64_t* active_bytes, int64_t* peak_bytes) {
  if (!sv) { set_error("NULL server"); return COLLO_ERR_INVALID_ARG; }
  if (active_bytes) *active_bytes = sv->active_bytes;
  if (peak_bytes) *peak_bytes = sv->peak_bytes;
  return COLLO_OK;
}

static bool valid_schedule(const collo_schedule* s) {
  return s && (s->big_threads == 256 || s->big_threads == 512) &&
         (s->slab_pairs == 8 || s->slab_pairs == 16) && s->solve_top_blocks >= 1 &&
         s->solve_top_blocks <= 4096 && s->solve_elems_per_block >= 1 &&
         s->solve_elems_per_block <= 1024;
}

collo_status collo_get_schedule(collo_schedule* out) {
  if (!out) { set_error("NULL argument"); return COLLO_ERR_INVALID_ARG; }
  std::memset(out, 0, sizeof(*out));
  const Schedule& g = schedule();
  out->big_threads = g.big_threads;
  out->slab_pairs = g.slab_pairs;
  out->solve_top_blocks = g.solve_top;
  out->solve_elems_per_block = g.solve_elems;
  return COLLO_OK;
}

collo_status collo_set_schedule(const collo_schedule* s) {
  if (!valid_schedule(s)) { set_error("bad schedule"); return COLLO_ERR_INVALID_ARG; }
  Schedule& g = schedule();
  g.big_threads = s->big_threads;
  g.slab_pairs = s->slab_pairs;
  g.solve_top = s->solve_top_blocks;
  g.solve_elems = s->solve_elems_per_block;
  return COLLO_OK;
}

collo_status collo_autotune(collo_problem* const* probs, int count, int precision, int reps,
                            collo_schedule* best, double* ms_before, double* ms_after) {
  if (!probs || count < 1 || reps < 1 || !best ||
      (precision != COLLO_PRECISION_FP64 && precision != COLLO_PRECISION_MIXED)) {
    set_error("bad argument");
    return COLLO_ERR_INVALID_ARG;
  }
  collo_schedule cur;
  collo_get_schedule(&cur);
  // the large-element kernel (phase 6) and the solve (phase 2) are timed
  // apart: their knobs do not interact
  auto timed = [&](const collo_schedule& c, int phase, double* ms) -> collo_status {
    collo_status s = collo_set_schedule(&c);
    if (s != COLLO_OK) return s;
    return collo_batch_time_phase(probs, count, phase, precision, reps, ms);
  };
  double f0 = 0, s0 = 0;
  collo_status st;
  if ((st = timed(cur, 6, &f0)) != COLLO_OK) { collo_set_schedule(&cur); return st; }
  if ((st = timed(cur, 2, &s0)) != COLLO_OK) { collo_set_schedule(&cur); return st; }
  collo_schedule b = cur;
  double fb = f0, sb = s0;
  for (int bt : {256, 512})
    for (int sp : {8, 16}) {
      collo_schedule c = b;
      c.big_threads = bt;
      c.slab_pairs = sp;
      double ms = 0;
      if ((st = timed(c, 6, &ms)) != COLLO_OK) { collo_set_schedule(&cur); return st; }
      if (ms < fb) { fb = ms; b.big_threads = bt; b.slab_pairs = sp; }
    }
  for (int top : {2, 4, 8, 16, 32})
    for (int per : {4, 8, 16, 32}) {
      collo_schedule c = b;
      c.solve_top_blocks = top;
      c.solve_elems_per_block = per;
      double ms = 0;
      if ((st = timed(c, 2, &ms)) != COLLO_OK) { collo_set_schedule(&cur); return st; }
      if (ms < sb) { sb = ms; b.solve_top_blocks = top; b.solve_elems_per_block = per; }
    }
  collo_set_schedule(&b);
  *best = b;
  if (ms_before) *ms_before = f0 + s0;
  if (ms_after) *ms_after = fb + sb;
  return COLLO_OK;
}

collo_status collo_server_counters(collo_server* sv, long long* newton_steps, long long* finished,
                                   long long* converged) {
  if (!sv) { set_error("NULL server"); return COLLO_ERR_INVALID_ARG; }
  if (newton_steps) *newton_steps = sv->newton_steps;
  if (finished) *finished = sv->finished;
  if (converged) *converged = sv->converged;
  return COLLO_OK;
}

collo_status collo_problem_set_wait_limit(collo_problem* prob, long long max_polls,
                                          int unreachable) {
  if (!prob || max_polls < 0) { set_error("bad argument"); return COLLO_ERR_INVALID_ARG; }
  COLLO_CUDA(cudaSetDevice(prob->device));
  prob->wait_polls = max_polls;
  prob->wait_unreachable = unreachable ? 1 : 0;
  if (prob->self) return prob->self->set_wait(prob->wait_polls, prob->wait_unreachable);
  return COLLO_OK;
}

collo_status collo_server_set_admission(collo_server* sv, int min_free_slots) {
  if (!sv || min_free_slots < 1) { set_error("bad argument"); return COLLO_ERR_INVALID_ARG; }
  sv->admit_min = min_free_slots;
  return COLLO_OK;
}

void* collo_server_stream(collo_server* sv) { return sv ? (void*)sv->R.stream : nullptr; }

collo_status collo_server_poll(collo_server* sv, long long ticket, collo_result* res) {
  if (!sv || !res) { set_error("bad argument"); return COLLO_ERR_INVALID_ARG; }
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) { set_error("unknown ticket"); return COLLO_ERR_INVALID_ARG; }
  auto* j = it->second;
  if (!j->done) return COLLO_PENDING;
  double* th = res->theta;
  *res = j->res;
  res->theta = th;
  if (th && j->prob->P.p) {
    const size_t nz = (size_t)j->prob->n_x - j->prob->P.p;
    COLLO_CUDA(cudaMemcpy(th, j->prob->x + nz, j->prob->P.p * sizeof(double), cudaMemcpyDefault));
  }
  return COLLO_OK;
}

void collo_server_destroy(collo_server* sv) {
  if (!sv) return;
  cudaSetDevice(sv->R.device);
  cudaStreamSynchronize(sv->R.stream);
  delete sv;
}

}  // extern "C"

collo_problem::~collo_problem() {
  delete self;
  collo::lifted_free(lifted);
}
