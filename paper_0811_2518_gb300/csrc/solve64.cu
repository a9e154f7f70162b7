// solve64.cu -- plain FP64 synchronous GaBP (Algorithm 2, broadcast form) on the GPU.
//
// Notation (paper, Algorithm 2 and eqs. eq_prec / eq_prec_message / eq_mean_message):
//   P~_i = A_ii + sum_{k in N(i)} P_ki,    h~_i = b_i + sum_{k in N(i)} h_ki,
//   P_ij = -A_ij^2 / (P~_i - P_ji),        h_ij = P_ij mu_ij = -A_ij (h~_i - h_ji) / (P~_i - P_ji),
//   x_i  = h~_i / P~_i                     (marginal mean, Algorithm 1 step 4).
// Messages are kept in information form (P, h = P mu); mu_ij of the paper is h_ij / P_ij.
//
// Round t of the parallel schedule reads round t-1 only (two message stores that
// swap roles, paper Sec. "The Gaussian BP Algorithm", scheduling paragraph):
//   in-message k -> i at t  =  f(A_ik, node record of k at t-1, reverse message i -> k at t-1).
// The in-messages of row i live in its slots; the reverse message is fetched from
// row k's slot, and the new node record of i is the sum over its row.  The same
// pass forms r_i = b_i - sum_j A_ij x_j^{(t-1)} from the node records it has
// gathered anyway, so the residual of round t-1's iterate costs one FMA per slot;
// the stop rule therefore decides about x^{(t-1)} during round t.
//
// Layout (Sell64): rows are ordered by degree inside windows of kSellWindow rows
// and cut into slices of 32; one warp runs a slice, one lane a row, and slot j of
// the slice's rows is one contiguous 32-wide line.  The round is bound by the FP64
// pipe (a Newton reciprocal and ~12 FP64 operations per slot on GB300's narrow FP64
// units), so what matters is that every lane of every FP64 instruction does work:
// rows of equal degree share a warp, and the row epilogue runs on all 32 lanes.
#include "gabp_internal.cuh"
#include "devutil.cuh"
#include "cluster.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

namespace gabp {

constexpr int kSellWindow = 4096;  // rows sorted by degree within windows of this many (a multiple of 32)

// Slots per lane whose loads the FP64 node round issues together, and the blocks per SM its
// register budget is sized for (__launch_bounds__).  Measured on the 2^20 random graph: 2 slots and
// 3 blocks (24 warps per SM) 0.558 ms per round; 4 blocks (64 registers) 0.589; 2 blocks 0.73;
// 1 slot with 4 blocks 0.633; 4 slots with 2 blocks 0.678.
#ifndef GABP_K64_UNROLL
#define GABP_K64_UNROLL 2
#endif
#ifndef GABP_K64_MINB
#define GABP_K64_MINB 3
#endif
constexpr int kU64 = GABP_K64_UNROLL;

struct Args64 {
  int n;
  int ns;                          // slices of 32 rows
  int Es;                          // sliced positions
  const int *__restrict__ srow;    // [ns * 32] row of each slice lane (-1 past n)
  const int *__restrict__ sp;      // [ns + 1] first position of each slice
  const int *__restrict__ sci;     // [Es] sender of each position (-1: padding)
  const int *__restrict__ srev;    // [Es] position of the reverse edge
  const double *__restrict__ sav;  // [Es] A_ik
  const double *__restrict__ ad;   // [n] A_ii
  double2 *M0, *M1;
  NodeRec64 *N0, *N1;
  DevCtl *ctl;
  double *partials;
  double *C;   // [Es] frozen coefficients (freeze != 0)
  int freeze;  // options.freeze_precisions on a plain node solve
  int wide;    // plain node rounds of a matrix of long rows: k64_wide
};

// Warp / lane of the calling thread and the number of warps in the grid.
struct WarpPos {
  int lane, warp, nwarps;
};
__device__ __forceinline__ WarpPos warp_pos() {
  return WarpPos{(int)(threadIdx.x & 31), (int)((blockIdx.x * kBlock + threadIdx.x) >> 5),
                 (int)((gridDim.x * kBlock) >> 5)};
}

// Round bookkeeping shared by the FP64 round kernels: this round checked
// x^{(t-1)} with squared residual rr; 'bad' counts zero cavities / precisions
// met while computing round t.
// The stopping parameters of a run, read once by a kernel that decides every round itself.
struct StopRule {
  double tol2bb;
  double *hist;
  int hist_cap, no_stop, check_from, max_iter;
};
__device__ __forceinline__ StopRule stop_rule(const DevCtl *ctl) {
  return StopRule{ctl->tol2bb, ctl->hist, ctl->hist_cap, ctl->no_stop, ctl->check_from, ctl->max_iter};
}
// decide64's decision alone: 1 when round t's sums end the run
__device__ __forceinline__ int stops64(const StopRule &q, int t, double rr, double bad) {
  const int tchk = t - 1;
  if (q.no_stop) return 0;
  return (tchk >= q.check_from && isfinite(rr) && rr <= q.tol2bb) || !isfinite(rr) ||
         (bad > 0.0 && t <= q.max_iter) || tchk >= q.max_iter;
}

// Records round t's residual and decision in the control block, with the stopping
// parameters q (stores only).  FENCE: a kernel whose other blocks read the decision after a
// grid barrier of its own publishes it with a device-scope fence; a cluster kernel's barrier
// orders it already.
template <bool FENCE = true>
__device__ __forceinline__ void record64(DevCtl *ctl, const StopRule &q, int t, double rr, double bad) {
  const int tchk = t - 1;
  ctl->round = t;
  if (q.hist && tchk < q.hist_cap) {  // residual of iterate tchk, before any decision
    q.hist[tchk] = rr;
    ctl->hist_len = tchk + 1;
  }
  if (q.no_stop) {
    ctl->rr = rr;
  } else if (tchk >= q.check_from && isfinite(rr) && rr <= q.tol2bb) {
    ctl->status = GABP_OK;
    ctl->iters = tchk;
    ctl->result_round = tchk;
    ctl->rr = rr;
    ctl->done = 1;
  } else if (!isfinite(rr)) {
    ctl->status = GABP_DIVERGED;
    ctl->iters = tchk;
    ctl->result_round = tchk;
    ctl->rr = rr;
    ctl->done = 1;
  } else if (bad > 0.0 && t <= q.max_iter) {
    ctl->status = GABP_BREAKDOWN;
    ctl->iters = t;
    ctl->result_round = tchk;
    ctl->rr = rr;
    ctl->done = 1;
  } else if (tchk >= q.max_iter) {
    ctl->status = GABP_NOT_CONVERGED;
    ctl->iters = tchk;
    ctl->result_round = tchk;
    ctl->rr = rr;
    ctl->done = 1;
  } else {
    ctl->rr = rr;
  }
  ctl->arrive = 0;
  if (FENCE) __threadfence();
}

// The same for a kernel that reads the stopping parameters from the control block each round.
__device__ __forceinline__ void decide64(DevCtl *ctl, int t, double rr, double bad) {
  record64<true>(ctl, stop_rule(ctl), t, rr, bad);
}

// Load flavours of the plain round body: the launch-per-round kernel streams its slot
// lines (evict first); the cooperative kernel reads data other blocks wrote through L2
// only and the read-only layout through the non-coherent path (L1 is not invalidated
// across its grid barrier).
template <bool COOP> __device__ __forceinline__ int ld_idx(const int *p) { return COOP ? __ldg(p) : __ldcs(p); }
template <bool COOP> __device__ __forceinline__ double ld_val(const double *p) { return COOP ? __ldg(p) : __ldcs(p); }
template <bool COOP> __device__ __forceinline__ double2 ld_msg(const double2 *p) { return COOP ? __ldcg(p) : __ldcs(p); }
template <bool COOP> __device__ __forceinline__ double ld_msgh(const double2 *p) {
  const double *q = reinterpret_cast<const double *>(p) + 1;
  return COOP ? __ldcg(q) : __ldcs(q);
}
template <bool COOP> __device__ __forceinline__ NodeRec64 ld_rec(const NodeRec64 *p) {
  if (!COOP) return *p;
  const double2 *r = reinterpret_cast<const double2 *>(p);
  const double2 q = __ldcg(r), q1 = __ldcg(r + 1);
  return NodeRec64{q.x, q.y, q1.x, q1.y};
}

// One slice of a plain round (node variant, no acceleration), a lane per row.
// MODE 0: Algorithm 2's round.  MODE 1 (freeze screen): the same, flagging rows whose
// P~_i moved since the previous round.  MODE 2 (freeze verify): the same, flagging
// precision messages that moved since the previous round (the slot's own previous
// message) and storing each slot's coefficient c = -A / (P~_k - P_ik) and each row's
// 1/P~ (the record's spare slot).  MODE 3 (frozen precisions): only the mean
// messages, h_ki = c (h~_k - h_ik), with the stored coefficients; P~ and 1/P~
// carried over.  All modes form x and the residual of the previous iterate as the
// round kernels do.
template <bool COOP, int MODE>
__device__ __forceinline__ void plain_slice(const Args64 &a, int sl, int lane, const double *__restrict__ b,
                                            const double2 *__restrict__ Min, double2 *__restrict__ Mout,
                                            const NodeRec64 *__restrict__ Nin, NodeRec64 *__restrict__ Nout,
                                            double &rr, int &bad, int &moving) {
  const int i = COOP ? __ldg(a.srow + sl * 32 + lane) : a.srow[sl * 32 + lane];
  const int q0 = COOP ? __ldg(a.sp + sl) : a.sp[sl];
  const int p0 = q0 + lane, wd = ((COOP ? __ldg(a.sp + sl + 1) : a.sp[sl + 1]) - q0) >> 5;
  double accP = 0.0, acch = 0.0, accr = 0.0;
  for (int j = 0; j < wd; j += kU64) {
    int k[kU64];
    double A[kU64], c[kU64], rh[kU64];
    double2 rv[kU64];
    NodeRec64 nk[kU64];
#pragma unroll
    for (int u = 0; u < kU64; ++u) {
      const int pos = p0 + 32 * (j + u);
      k[u] = j + u < wd ? ld_idx<COOP>(a.sci + pos) : -1;
      if (k[u] >= 0) {
        A[u] = ld_val<COOP>(a.sav + pos);
        const int rp = ld_idx<COOP>(a.srev + pos);
        if (MODE == 3) {
          c[u] = COOP ? __ldcg(a.C + pos) : __ldcs(a.C + pos);  // written by this launch when COOP
          rh[u] = ld_msgh<COOP>(Min + rp);  // mean message i -> k of round t-1
        } else {
          rv[u] = ld_msg<COOP>(Min + rp);   // message i -> k of round t-1
          if (MODE == 2) rh[u] = ld_msg<COOP>(Min + pos).x;  // this slot's precision message at t-1
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU64; ++u)
      if (k[u] >= 0) nk[u] = ld_rec<COOP>(Nin + k[u]);  // node k at round t-1
#pragma unroll
    for (int u = 0; u < kU64; ++u) {
      if (k[u] < 0) continue;
      const int pos = p0 + 32 * (j + u);
      if (MODE == 3) {
        const double hn = __dmul_rn(c[u], nk[u].h - rh[u]);
        double *dst = reinterpret_cast<double *>(Mout + pos) + 1;
        if (COOP) *dst = hn; else __stcs(dst, hn);
        acch = __dadd_rn(acch, hn);
      } else {
        const double den = nk[u].P - rv[u].x;  // cavity precision P_{k\i}
        bad |= is_zero64(den);
        const double cin = -A[u] * rcp64(den);
        // the aggregates add the stored (rounded) messages, as Algorithm 2 sums them
        const double2 m = make_double2(__dmul_rn(cin, A[u]), __dmul_rn(cin, nk[u].h - rv[u].y));
        if (COOP) Mout[pos] = m; else __stcs(Mout + pos, m);
        if (MODE == 2) {
          moving |= ulp_apart(m.x, rh[u]);
          a.C[pos] = cin;
        }
        accP = __dadd_rn(accP, m.x);
        acch = __dadd_rn(acch, m.y);
      }
      accr = fma(A[u], nk[u].x, accr);
    }
  }
  if (i >= 0) {
    const double bi = COOP ? __ldg(b + i) : b[i], d = COOP ? __ldg(a.ad + i) : a.ad[i];
    const NodeRec64 own = ld_rec<COOP>(Nin + i);
    if (MODE == 3) {
      const double h = bi + acch;
      Nout[i] = NodeRec64{own.P, h, h * own.pad, own.pad};
    } else {
      const double P = d + accP, h = bi + acch;
      bad |= is_zero64(P);
      if (MODE == 1) moving |= ulp_apart(P, own.P);
      const double ip = rcp64(P);
      Nout[i] = NodeRec64{P, h, h * ip, MODE == 2 ? ip : h * ip};
    }
    const double r = bi - fma(d, own.x, accr);
    rr = fma(r, r, rr);
  }
}

// Round 0 (Algorithm 1/2 step 1): all messages zero, so P~_i = A_ii, h~_i = b_i.
// Warm start (warm = 1): round 0 takes the messages already in M0 (a previous
// solve's, or imported ones) and forms the aggregates from them with this b:
// any starting messages lead to the same fixed point when the iteration converges.
__global__ void __launch_bounds__(kBlock) k64_init(Args64 a, double tol, int max_iter, int warm) {
  const double *b = a.ctl->b;
  const WarpPos w = warp_pos();
  double bb = 0.0;
  for (int sl = w.warp; sl < a.ns; sl += w.nwarps) {
    const int i = a.srow[sl * 32 + w.lane];
    if (i < 0) continue;
    double bi = b[i], d = a.ad[i], P = d, h = bi;
    if (warm) {
      const int p0 = a.sp[sl], wd = (a.sp[sl + 1] - p0) >> 5;
      for (int j = 0; j < wd; ++j) {
        const int pos = p0 + 32 * j + w.lane;
        if (a.sci[pos] < 0) break;
        const double2 m = a.M0[pos];
        P += m.x;
        h += m.y;
      }
    }
    const double x0 = h / P;
    a.N0[i] = NodeRec64{P, h, x0, x0};  // y^(0) = x^(0)
    bb = fma(bi, bi, bb);
  }
  double v[1] = {bb}, tot[1];
  const int modes[1] = {0};
  block_sum<1>(v);
  if (last_block_reduce<1>(v, modes, a.partials, &a.ctl->arrive, tot) && threadIdx.x == 0) {
    DevCtl *c = a.ctl;
    c->round = 0;
    c->bb = tot[0];
    c->tol2bb = tol * tol * tot[0];
    c->max_iter = max_iter;
    c->check_from = 1;
    c->stable = 0;
    c->edge_bad = 0;
    c->rr = tot[0];
    c->arrive = 0;
    if (tot[0] == 0.0) {  // b = 0: x = 0 after no round
      c->done = 1;
      c->status = GABP_OK;
      c->iters = 0;
      c->result_round = 0;
      c->rr = 0.0;
    } else {
      c->done = 0;
      c->status = GABP_NOT_CONVERGED;
      c->iters = 0;
      c->result_round = 0;
    }
    __threadfence();
  }
}

// Aitken's extrapolation (Sec. "Convergence Acceleration") of one node's last
// three marginal means x0 = x^(t-2), x1 = x^(t-1), x2 = x^(t):
// y = x0 - (x1 - x0)^2 / (x2 - 2 x1 + x0), or x2 where the second difference is
// negligible (|D| <= 1e-14 |x2|: the node has stopped moving).
__device__ __forceinline__ double aitken64(double x0, double x1, double x2) {
  const double D = x2 - 2.0 * x1 + x0;
  if (!(fabs(D) > 1e-14 * fabs(x2))) return x2;
  const double d = x1 - x0;
  return x0 - d * d / D;
}

// Acceleration modes of the FP64 node round (options.accel).
enum { ACC_NONE = 0, ACC_AITKEN = 1, ACC_STEFFENSEN = 2 };

// One plain round over this kernel's slices in mode MODE of plain_slice, then the
// block sums and, in the last block, the freeze state's step and the decision.
template <int MODE>
__device__ __forceinline__ void plain_round(const Args64 &a, DevCtl *ctl, int t, const double *__restrict__ b,
                                            const double2 *__restrict__ Min, double2 *__restrict__ Mout,
                                            const NodeRec64 *__restrict__ Nin, NodeRec64 *__restrict__ Nout,
                                            const WarpPos &w) {
  double rr = 0.0;
  int bad = 0, moving = 0;
  for (int sl = w.warp; sl < a.ns; sl += w.nwarps)
    plain_slice<false, MODE>(a, sl, w.lane, b, Min, Mout, Nin, Nout, rr, bad, moving);
  constexpr int NV = MODE > 0 ? 3 : 2;  // the moving count only when the freeze is on
  double v[NV], tot[NV];
  int modes[NV];
  v[0] = rr;
  v[1] = (double)bad;
  if constexpr (NV > 2) v[2] = (double)moving;
  for (int q = 0; q < NV; ++q) modes[q] = 0;
  block_sum<NV>(v);
  if (last_block_reduce<NV>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    if constexpr (MODE > 0) freeze_step(ctl, MODE - 1, t, tot[2]);
    decide64(ctl, t, tot[0], tot[1]);
  }
}

// The plain round for long rows (Algorithm 2's round, as plain_slice's mode 0): a warp
// per row of the sliced layout, its lanes on the row's slots j, j + 32, ... (slot j
// of slice row r is sp[s] + 32 j + r), the aggregates and the residual term reduced
// across the warp, the row's epilogue on lane 0.  A layout with one lane per row
// gives a matrix of few long rows (dense ones) only n / 32 warps.
__global__ void __launch_bounds__(kBlock) k64_wide(Args64 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int t = ctl->round + 1;
  const double *__restrict__ b = ctl->b;
  const double2 *__restrict__ Min = (t & 1) ? a.M0 : a.M1;
  double2 *__restrict__ Mout = (t & 1) ? a.M1 : a.M0;
  const NodeRec64 *__restrict__ Nin = (t & 1) ? a.N0 : a.N1;
  NodeRec64 *__restrict__ Nout = (t & 1) ? a.N1 : a.N0;
  const WarpPos w = warp_pos();
  double rr = 0.0;
  int bad = 0;
  for (int q = w.warp; q < a.ns * 32; q += w.nwarps) {
    const int i = a.srow[q];
    if (i < 0) continue;  // warp-uniform
    const int sl = q >> 5, r = q & 31;
    const int p0 = a.sp[sl] + r, wd = (a.sp[sl + 1] - a.sp[sl]) >> 5;
    double accP = 0.0, acch = 0.0, accr = 0.0;
    for (int j = w.lane; j < wd; j += 32) {
      const int pos = p0 + 32 * j;
      const int k = __ldcs(a.sci + pos);
      if (k < 0) continue;
      const double A = __ldcs(a.sav + pos);
      const double2 rv = __ldcs(Min + __ldcs(a.srev + pos));  // message i -> k of round t-1
      const NodeRec64 nk = Nin[k];                              // node k at round t-1
      const double den = nk.P - rv.x;
      bad |= is_zero64(den);
      const double cin = -A * rcp64(den);
      const double2 m = make_double2(__dmul_rn(cin, A), __dmul_rn(cin, nk.h - rv.y));
      __stcs(Mout + pos, m);
      accP = __dadd_rn(accP, m.x);
      acch = __dadd_rn(acch, m.y);
      accr = fma(A, nk.x, accr);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      accP += __shfl_xor_sync(0xffffffffu, accP, o);
      acch += __shfl_xor_sync(0xffffffffu, acch, o);
      accr += __shfl_xor_sync(0xffffffffu, accr, o);
    }
    if (w.lane == 0) {
      const double bi = b[i], d = a.ad[i];
      const NodeRec64 own = Nin[i];
      const double P = d + accP, h = bi + acch;
      bad |= is_zero64(P);
      const double ip = rcp64(P);
      Nout[i] = NodeRec64{P, h, h * ip, h * ip};
      const double rres = bi - fma(d, own.x, accr);
      rr = fma(rres, rres, rr);
    }
  }
  double v[2] = {rr, (double)bad}, tot[2];
  const int modes[2] = {0, 0};
  block_sum<2>(v);
  if (last_block_reduce<2>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) decide64(ctl, t, tot[0], tot[1]);
}

// The plain round with the precision freeze on: MODE 1 (screen), 2 (verify and store)
// or 3 (frozen).  A round launches k64_frz<3>, <2>, <1> in that order and each
// returns unless the freeze state is MODE - 1.  The state only grows by one step at
// a time, except that a failed verification returns it to 0: so one of the three
// runs, or k64_frz<2> and then k64_frz<1> (two rounds; the round count and the stop
// rule live on the device, so a launch slot may hold two rounds).
template <int MODE>
__global__ void __launch_bounds__(kBlock, GABP_K64_MINB) k64_frz(Args64 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done || ctl->fstate != MODE - 1) return;
  const int t = ctl->round + 1;
  const double2 *__restrict__ Min = (t & 1) ? a.M0 : a.M1;
  double2 *__restrict__ Mout = (t & 1) ? a.M1 : a.M0;
  const NodeRec64 *__restrict__ Nin = (t & 1) ? a.N0 : a.N1;
  NodeRec64 *__restrict__ Nout = (t & 1) ? a.N1 : a.N0;
  plain_round<MODE>(a, ctl, t, ctl->b, Min, Mout, Nin, Nout, warp_pos());
}

// Fused node-centric round (GABP_VARIANT_NODE): a warp per slice, a lane per row.
// ACC = ACC_AITKEN: every node also forms y^(t) = aitken(x^(t-2), x^(t-1), x^(t))
// into its record's spare slot (x^(t-2) is the record being overwritten), and the
// fused stop rule takes the residual of y^(t-1) instead of x^(t-1).
// ACC = ACC_STEFFENSEN (Steffensen's iterations, Sec. "Convergence Acceleration"):
// rounds pair into cycles (t odd: first round, t even: second).  The first round
// keeps the cycle's starting iterate x_n in the spare slot; the second also sums
// <d, D> and <D, D> (d = x_{n+2} - x_{n+1}, D = x_{n+2} - 2 x_{n+1} + x_n), whose
// quotient, the scalar step lam, its last block stores for k64_steff.
template <int ACC>
__global__ void __launch_bounds__(kBlock, GABP_K64_MINB) k64_node(Args64 a) {
  constexpr bool AIT = ACC == ACC_AITKEN;
  constexpr bool STF = ACC == ACC_STEFFENSEN;
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int t = ctl->round + 1;
  const double *__restrict__ b = ctl->b;
  const double2 *__restrict__ Min = (t & 1) ? a.M0 : a.M1;  // round t-1
  double2 *__restrict__ Mout = (t & 1) ? a.M1 : a.M0;       // round t
  const NodeRec64 *__restrict__ Nin = (t & 1) ? a.N0 : a.N1;
  NodeRec64 *__restrict__ Nout = (t & 1) ? a.N1 : a.N0;
  const WarpPos w = warp_pos();
  if (ACC == ACC_NONE) {
    plain_round<0>(a, ctl, t, b, Min, Mout, Nin, Nout, w);
    return;
  }
  double rr = 0.0, sdD = 0.0, sDD = 0.0;
  int bad = 0;
  for (int sl = w.warp; sl < a.ns; sl += w.nwarps) {
    const int i = a.srow[sl * 32 + w.lane];
    const int p0 = a.sp[sl] + w.lane, wd = (a.sp[sl + 1] - a.sp[sl]) >> 5;
    double accP = 0.0, acch = 0.0, accr = 0.0;
    // kU64 slots per lane per step, their loads issued before use; the slot lines and the
    // reverse messages are read once per round (streaming), the sender records are the
    // reused working set
    for (int j = 0; j < wd; j += kU64) {
      int k[kU64];
      double A[kU64];
      double2 rv[kU64];
      NodeRec64 nk[kU64];
#pragma unroll
      for (int u = 0; u < kU64; ++u) {
        const int pos = p0 + 32 * (j + u);
        k[u] = j + u < wd ? __ldcs(a.sci + pos) : -1;
        if (k[u] >= 0) {
          A[u] = __ldcs(a.sav + pos);
          rv[u] = __ldcs(Min + __ldcs(a.srev + pos));  // message i -> k of round t-1
        }
      }
#pragma unroll
      for (int u = 0; u < kU64; ++u)
        if (k[u] >= 0) nk[u] = Nin[k[u]];  // node k at round t-1
#pragma unroll
      for (int u = 0; u < kU64; ++u) {
        if (k[u] >= 0) {
          const double den = nk[u].P - rv[u].x;  // cavity precision P_{k\i}
          bad |= is_zero64(den);
          const double cin = -A[u] * rcp64(den);
          // the aggregates add the stored (rounded) messages, as Algorithm 2 sums them: no
          // contraction of a product into the sum
          const double2 m = make_double2(__dmul_rn(cin, A[u]), __dmul_rn(cin, nk[u].h - rv[u].y));
          __stcs(Mout + p0 + 32 * (j + u), m);
          accP = __dadd_rn(accP, m.x);
          acch = __dadd_rn(acch, m.y);
          accr = fma(A[u], AIT ? nk[u].pad : nk[u].x, accr);
        }
      }
    }
    if (i >= 0) {
      const double bi = b[i], d = a.ad[i];
      const double P = d + accP, h = bi + acch;
      bad |= is_zero64(P);
      const NodeRec64 own = Nin[i];
      const double xt = h * rcp64(P);
      double yt = xt;
      if (AIT && t >= 2) yt = aitken64(Nout[i].x, own.x, xt);
      if (STF) {
        if (!(t & 1)) {  // own.x = x_{n+1}, own.pad = x_n
          const double dd = xt - own.x, D = dd - (own.x - own.pad);
          sdD = fma(dd, D, sdD);
          sDD = fma(D, D, sDD);
        }
        yt = own.x;  // after a first round: x_n, the cycle's starting iterate
      }
      Nout[i] = NodeRec64{P, h, xt, yt};
      const double r = bi - fma(d, AIT ? own.pad : own.x, accr);
      rr = fma(r, r, rr);
    }
  }
  if (STF) {
    double v[4] = {rr, (double)bad, sdD, sDD}, tot[4];
    const int modes[4] = {0, 0, 0, 0};
    block_sum<4>(v);
    if (last_block_reduce<4>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) {
      if (!(t & 1)) {  // the cycle's scalar step; 0 where nothing moves or the quotient is not finite
        const double lam = tot[3] > 0.0 ? tot[2] / tot[3] : 0.0;
        ctl->lam = isfinite(lam) ? lam : 0.0;
      }
      decide64(ctl, t, tot[0], tot[1]);
    }
    return;
  }
  double v[2] = {rr, (double)bad}, tot[2];
  const int modes[2] = {0, 0};
  block_sum<2>(v);
  if (last_block_reduce<2>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0)
    decide64(ctl, t, tot[0], tot[1]);
}

// Small and medium graphs (at most kCoopMaxSlices slices): every round of a plain
// solve (node variant) in ONE cooperative launch of small blocks spread over many
// SMs.  Per round: the same per-row arithmetic and decision as k64_node<ACC_NONE>;
// then a grid barrier whose last arriving block sums the blocks' partials (in block
// order) and takes the decision before it releases the others.  At these sizes a
// round is a few dependent memory accesses plus little FP64 work per SM (GB300 retires
// 2 FP64 operations per SM and clock, so the work must stay spread: one block running
// every round measured slower than a launch per round), and the launch and the
// separate reduction per round would cost more than the round.  Data written by other
// blocks (messages, records, control block) is read through L2 only (__ldcg: L1 is not
// invalidated across the barrier); the layout and A are read-only for the whole launch.
// The barrier's wait is bounded (kCoopBarrierLimit clock cycles, ~2 s; all blocks are
// co-resident, so it always completes): if it ever gave up, the kernel raises *err and
// every block returns.  The loop is bounded by max_rounds.
#ifndef GABP_COOP_THREADS
#define GABP_COOP_THREADS 64
#endif
#ifndef GABP_COOP_SLEEP
#define GABP_COOP_SLEEP 32
#endif
constexpr int kCoopThreads = GABP_COOP_THREADS;
constexpr int kCoopMaxSlices = 4096;
constexpr long long kCoopBarrierLimit = 4000000000LL;

template <bool FRZ>
__global__ void __launch_bounds__(kCoopThreads, FRZ ? 8 : 0) k64_coop(Args64 a, unsigned *bar, int *err, int max_rounds) {
  DevCtl *ctl = a.ctl;
  __shared__ int s_last, s_go;
  __shared__ unsigned s_gen;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kCoopThreads + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kCoopThreads) >> 5;
  const double *__restrict__ b = ctl->b;
  for (int iter = 0; iter < max_rounds; ++iter) {
    const int t = __ldcg(&ctl->round) + 1;
    const int fs = FRZ ? __ldcg(&ctl->fstate) : -1;
    const double2 *__restrict__ Min = (t & 1) ? a.M0 : a.M1;
    double2 *__restrict__ Mout = (t & 1) ? a.M1 : a.M0;
    const NodeRec64 *__restrict__ Nin = (t & 1) ? a.N0 : a.N1;
    NodeRec64 *__restrict__ Nout = (t & 1) ? a.N1 : a.N0;
    double rr = 0.0;
    int bad = 0, moving = 0;
    for (int sl = warp; sl < a.ns; sl += nwarps) {
      if (!FRZ) plain_slice<true, 0>(a, sl, lane, b, Min, Mout, Nin, Nout, rr, bad, moving);
      else if (fs == 0) plain_slice<true, 1>(a, sl, lane, b, Min, Mout, Nin, Nout, rr, bad, moving);
      else if (fs == 1) plain_slice<true, 2>(a, sl, lane, b, Min, Mout, Nin, Nout, rr, bad, moving);
      else plain_slice<true, 3>(a, sl, lane, b, Min, Mout, Nin, Nout, rr, bad, moving);
    }
    // grid barrier; the last block to arrive reduces and decides
    constexpr int NV = FRZ ? 3 : 2;
    double v[NV];
    v[0] = rr;
    v[1] = (double)bad;
    if constexpr (FRZ) v[2] = (double)moving;
    block_sum_nt<NV, kCoopThreads>(v);
    if (threadIdx.x == 0) {
      a.partials[blockIdx.x] = v[0];
      a.partials[gridDim.x + blockIdx.x] = v[1];
      if constexpr (FRZ) a.partials[2 * gridDim.x + blockIdx.x] = v[2];
      const unsigned g = *(volatile unsigned *)(bar + 1);
      __threadfence();
      s_last = atomicAdd(bar, 1u) == gridDim.x - 1;
      s_gen = g;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      double w[NV];
      for (int q = 0; q < NV; ++q) w[q] = 0.0;
      for (int q = threadIdx.x; q < (int)gridDim.x; q += kCoopThreads) {
        w[0] += __ldcg(a.partials + q);
        w[1] += __ldcg(a.partials + gridDim.x + q);
        if constexpr (FRZ) w[2] += __ldcg(a.partials + 2 * gridDim.x + q);
      }
      block_sum_nt<NV, kCoopThreads>(w);
      if (threadIdx.x == 0) {
        if constexpr (FRZ) freeze_step(ctl, fs, t, w[2]);
        decide64(ctl, t, w[0], w[1]);
        s_go = !ctl->done;
        bar[0] = 0;
        __threadfence();
        atomicAdd(bar + 1, 1u);
      }
    } else if (threadIdx.x == 0) {
      volatile unsigned *gen = bar + 1;
      const long long t0 = clock64();
      int ok = 1;
      while (*gen == s_gen) {
        if (*(volatile int *)err || clock64() - t0 > kCoopBarrierLimit) { ok = 0; break; }
        if (GABP_COOP_SLEEP) __nanosleep(GABP_COOP_SLEEP);
      }
      if (!ok) atomicExch(err, 1);
      __threadfence();
      s_go = ok && !__ldcg(&ctl->done);
    }
    __syncthreads();
    if (!s_go) break;
  }
}

// Every plain round of a small graph in one thread-block cluster (up to 16 CTAs of NW
// warps, one SM each, a slice per warp): the cluster's hardware barrier replaces the
// grid barrier.  Per round every warp posts its residual sum in its CTA's shared
// memory; after the cluster barrier every warp fetches all posts (distributed shared
// memory), adds them the same way and takes the same decision, so all CTAs leave after
// the same round (no wait can be left open) and CTA 0 records it.  Data written by
// other CTAs is read through L2 (plain_slice's cooperative flavour); the barrier
// releases and acquires at cluster scope.  Two warps a CTA up to 32 slices; four (all
// four schedulers of the SM, each with its own FP64 unit) up to 64; eight (two a
// scheduler) up to 128 when no slice is wider than kCluster8MaxWidth slots a row: two warps share
// each FP64 unit, so the widest slices set the round (64x64 grid, width 4: 7.9 us per round against
// 10.2 with the cooperative grid; 4096-row random graph of degree 4, width up to ~16: 19.9 against
// 18.7).
constexpr int kClusterMax = 16;
#ifndef GABP_CLUSTER_MAX_SLICES
#define GABP_CLUSTER_MAX_SLICES 128
#endif
// Two warps a CTA up to this many slices, four above.  Four from the start: 32x32 grid 4.69 against
// 4.53 us per round (8x8: 4.00 against 4.22).
#ifndef GABP_CLUSTER_NW2_MAX_SLICES
#define GABP_CLUSTER_NW2_MAX_SLICES 32
#endif
// Slots per lane whose loads the on-chip round issues together: 4 against 2, 32x32 grid 4.44 against
// 4.53 us per round, 2048-row random graph 13.2 against 13.4, 1280-row 15.1 against 14.95.
#ifndef GABP_CHIP_UNROLL
#define GABP_CHIP_UNROLL 4
#endif
constexpr int kUChip = GABP_CHIP_UNROLL;
constexpr int kClusterMaxSlices = GABP_CLUSTER_MAX_SLICES;
constexpr int kCluster8MaxWidth = 8;

template <bool FRZ, int NW>
__global__ void __launch_bounds__(32 * NW) k64_cluster(Args64 a, int max_rounds) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank(), csize = cl.num_blocks();
  __shared__ ClusterPart part[2][NW];  // [round parity][warp]
  DevCtl *ctl = a.ctl;
  const double *__restrict__ b = ctl->b;
  const int t0 = ctl->round;  // read by every CTA before the first barrier, written only after it
  const StopRule rule = stop_rule(ctl);  // CTA 0 writes none of these fields
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warp = (int)(rank * NW) + wib;
  const int nwarps = (int)(csize * NW);
  for (int iter = 0; iter < max_rounds; ++iter) {
    const int t = t0 + 1 + iter;
    const int fs = FRZ ? __ldcg(&ctl->fstate) : -1;  // written by CTA 0 before the last barrier
    const double2 *__restrict__ Min = (t & 1) ? a.M0 : a.M1;
    double2 *__restrict__ Mout = (t & 1) ? a.M1 : a.M0;
    const NodeRec64 *__restrict__ Nin = (t & 1) ? a.N0 : a.N1;
    NodeRec64 *__restrict__ Nout = (t & 1) ? a.N1 : a.N0;
    double rr = 0.0;
    int bad = 0, moving = 0;
    for (int sl = warp; sl < a.ns; sl += nwarps) {
      if (!FRZ) plain_slice<true, 0>(a, sl, lane, b, Min, Mout, Nin, Nout, rr, bad, moving);
      else if (fs == 0) plain_slice<true, 1>(a, sl, lane, b, Min, Mout, Nin, Nout, rr, bad, moving);
      else if (fs == 1) plain_slice<true, 2>(a, sl, lane, b, Min, Mout, Nin, Nout, rr, bad, moving);
      else plain_slice<true, 3>(a, sl, lane, b, Min, Mout, Nin, Nout, rr, bad, moving);
    }
    // flags: bit 0 a zero cavity or node precision, bit 1 a precision moved (the freeze's screen)
    const ClusterSums tot =
        cluster_sums<NW>(cl, part[t & 1], rr, (bad ? 1 : 0) | (moving ? 2 : 0), lane, wib, nwarps);
    const bool stop = stops64(rule, t, tot.rr, tot.flags & 1);
    if (rank == 0 && threadIdx.x == 0) {
      if constexpr (FRZ) freeze_step(ctl, fs, t, (tot.flags & 2) ? 1.0 : 0.0);
      record64<false>(ctl, rule, t, tot.rr, tot.flags & 1);
    }
    if (stop) break;
    if constexpr (FRZ) cl.sync();  // the freeze state CTA 0 wrote is read by every CTA next round
  }
  cl.sync();  // no CTA leaves while a peer may still read its shared memory
}

// The cluster rounds with the whole state in the cluster's shared memory, for graphs
// whose state fits: each CTA holds its own rows' records (both rounds'), b and A_ii,
// and its own slots' reverse references, values and messages (both rounds').  A slot
// reads the sender's record and the reverse message from the CTA that owns the sender
// -- the reverse slot sits in the sender's row, so one CTA holds both -- through
// distributed shared memory; everything a round writes stays in its own CTA, and the
// round's only global-memory traffic is the control block.  The slices, warps, lanes
// and sums are k64_cluster's, so every value is bitwise the same; the state is loaded
// from and written back to the global arrays (both parities) around the rounds.
struct ChipShape {
  int smax;  // own slots of the largest CTA
  int rmax;  // own rows (32 per own slice) of the largest CTA
};
__host__ __device__ inline size_t chip_bytes(const ChipShape &c, int ns) {
  return (size_t)48 * c.smax + (size_t)84 * c.rmax + (size_t)8 * ns + (size_t)128 * ns;
}
// a row's place in its owner CTA: slice s belongs to warp s mod (NW cs), i.e. CTA
// (s mod NW cs) / NW, which holds its slices in increasing order, 32 rows each
template <int NW>
__host__ __device__ __forceinline__ int chip_row_ref(int s, int lane, int nwarps) {
  const int o = (s % nwarps) / NW, q = NW * (s / nwarps) + (s % nwarps) % NW;
  return (o << 24) | (q * 32 + lane);
}

template <int NW>
__global__ void __launch_bounds__(32 * NW) k64_chip(Args64 a, ChipShape c, int max_rounds) {
  constexpr int NT = 32 * NW;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank(), csize = cl.num_blocks();
  extern __shared__ __align__(32) unsigned char smem[];
  NodeRec64 *R0 = reinterpret_cast<NodeRec64 *>(smem);  // own rows, by local row
  NodeRec64 *R1 = R0 + c.rmax;
  double2 *Ml0 = reinterpret_cast<double2 *>(R1 + c.rmax);  // own slots, by local slot
  double2 *Ml1 = Ml0 + c.smax;
  double *savl = reinterpret_cast<double *>(Ml1 + c.smax);
  double *bl = savl + c.smax;
  double *dl = bl + c.rmax;
  int *kref = reinterpret_cast<int *>(dl + c.rmax);  // sender: owner rank << 24 | its local row (-1: padding)
  int *rref = kref + c.smax;                         // reverse slot: owner rank << 24 | its local slot
  int *srowl = rref + c.smax;
  int2 *tab = reinterpret_cast<int2 *>(srowl + c.rmax);  // per slice: owner rank, local first slot
  int *inv = reinterpret_cast<int *>(tab + a.ns);        // per row: its slice position (set-up only)
  __shared__ ClusterPart part[2][NW];
  DevCtl *ctl = a.ctl;
  const double *__restrict__ b = ctl->b;
  const int t0 = ctl->round;
  const StopRule rule = stop_rule(ctl);  // CTA 0 writes none of these fields
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warp = (int)(rank * NW) + wib;
  const int nwarps = (int)(csize * NW);
  if (threadIdx.x == 0) {
    int base[kClusterMax];
    for (int r = 0; r < kClusterMax; ++r) base[r] = 0;
    for (int sl = 0; sl < a.ns; ++sl) {
      const int o = (sl % nwarps) / NW;
      tab[sl] = make_int2(o, base[o]);
      base[o] += a.sp[sl + 1] - a.sp[sl];
    }
  }
  for (int e = threadIdx.x; e < 32 * a.ns; e += NT) {
    const int i = a.srow[e];
    if (i >= 0) inv[i] = e;
  }
  __syncthreads();
  {
    int q = 0;  // own slice index
    for (int sl = 0; sl < a.ns; ++sl) {
      if ((int)tab[sl].x != (int)rank) continue;
      const int p0 = a.sp[sl], wd = (a.sp[sl + 1] - p0) >> 5, lb = tab[sl].y;
      for (int e = threadIdx.x; e < 32; e += NT) {
        const int i = a.srow[sl * 32 + e], lr = q * 32 + e;
        srowl[lr] = i;
        bl[lr] = i >= 0 ? b[i] : 0.0;
        dl[lr] = i >= 0 ? a.ad[i] : 0.0;
        if (i >= 0) {  // both parities, so the write-back returns what the rounds do not change
          R0[lr] = a.N0[i];
          R1[lr] = a.N1[i];
        }
      }
      for (int e = threadIdx.x; e < 32 * wd; e += NT) {
        const int pos = p0 + e, li = lb + e;
        const int k = a.sci[pos];
        savl[li] = a.sav[pos];
        Ml0[li] = a.M0[pos];
        Ml1[li] = a.M1[pos];
        int kr = -1, rr = 0;
        if (k >= 0) {
          const int ek = inv[k];
          kr = chip_row_ref<NW>(ek >> 5, ek & 31, nwarps);
          const int rp = a.srev[pos];
          int lo = 0, hi = a.ns - 1;  // the slice holding position rp
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.sp[mid] <= rp) lo = mid; else hi = mid - 1;
          }
          rr = (tab[lo].x << 24) | (tab[lo].y + (rp - a.sp[lo]));
        }
        kref[li] = kr;
        rref[li] = rr;
      }
      ++q;
    }
  }
  cl.sync();  // every CTA's state is in place before any peer reads it
  int ran = 0;
  for (int iter = 0; iter < max_rounds; ++iter) {
    const int t = t0 + 1 + iter;
    const NodeRec64 *Rin = (t & 1) ? R0 : R1;  // round t-1
    NodeRec64 *Rout = (t & 1) ? R1 : R0;
    double2 *Min = (t & 1) ? Ml0 : Ml1;
    double2 *Mout = (t & 1) ? Ml1 : Ml0;
    double rr = 0.0;
    int bad = 0;
    for (int sl = warp, qq = wib; sl < a.ns; sl += nwarps, qq += NW) {
      const int lb = tab[sl].y, wd = (a.sp[sl + 1] - a.sp[sl]) >> 5;
      const int lr = qq * 32 + lane, i = srowl[lr];
      double accP = 0.0, acch = 0.0, accr = 0.0;
      for (int j = 0; j < wd; j += kUChip) {
        int kr[kUChip];
        double A[kUChip];
        double2 rv[kUChip];
        NodeRec64 nk[kUChip];
#pragma unroll
        for (int u = 0; u < kUChip; ++u) {
          const int li = lb + 32 * (j + u) + lane;
          kr[u] = j + u < wd ? kref[li] : -1;
          if (kr[u] >= 0) {
            A[u] = savl[li];
            const int ref = rref[li];
            rv[u] = *cl.map_shared_rank(Min + (ref & 0xffffff), (unsigned)(ref >> 24));  // message i -> k at t-1
            nk[u] = *cl.map_shared_rank(Rin + (kr[u] & 0xffffff), (unsigned)(kr[u] >> 24));  // node k at t-1
          }
        }
#pragma unroll
        for (int u = 0; u < kUChip; ++u) {
          if (kr[u] < 0) continue;
          const double den = nk[u].P - rv[u].x;
          bad |= is_zero64(den);
          const double cin = -A[u] * rcp64(den);
          const double2 m = make_double2(__dmul_rn(cin, A[u]), __dmul_rn(cin, nk[u].h - rv[u].y));
          Mout[lb + 32 * (j + u) + lane] = m;
          accP = __dadd_rn(accP, m.x);
          acch = __dadd_rn(acch, m.y);
          accr = fma(A[u], nk[u].x, accr);
        }
      }
      if (i >= 0) {
        const double bi = bl[lr], d = dl[lr];
        const NodeRec64 own = Rin[lr];
        const double P = d + accP, h = bi + acch;
        bad |= is_zero64(P);
        const double ip = rcp64(P);
        Rout[lr] = NodeRec64{P, h, h * ip, h * ip};
        const double res = bi - fma(d, own.x, accr);
        rr = fma(res, res, rr);
      }
    }
    ++ran;
    const ClusterSums tot = cluster_sums<NW>(cl, part[t & 1], rr, bad, lane, wib, nwarps);
    if (rank == 0 && threadIdx.x == 0) record64<false>(ctl, rule, t, tot.rr, tot.flags & 1);
    if (stops64(rule, t, tot.rr, tot.flags & 1)) break;
  }
  // back to the global arrays, both parities: the own slots' messages and the own rows' records
  // (rounds run: the last wrote after its barrier's arrival of every warp, read here after it)
  if (ran > 0) {
    int q = 0;
    for (int sl = 0; sl < a.ns; ++sl) {
      if ((int)tab[sl].x != (int)rank) continue;
      const int p0 = a.sp[sl], wd = (a.sp[sl + 1] - p0) >> 5, lb = tab[sl].y;
      for (int e = threadIdx.x; e < 32 * wd; e += NT) {
        a.M0[p0 + e] = Ml0[lb + e];
        a.M1[p0 + e] = Ml1[lb + e];
      }
      for (int e = threadIdx.x; e < 32; e += NT) {
        const int i = srowl[q * 32 + e];
        if (i >= 0) {
          a.N0[i] = R0[q * 32 + e];
          a.N1[i] = R1[q * 32 + e];
        }
      }
      ++q;
    }
  }
  cl.sync();  // no CTA leaves while a peer may still read its shared memory
}

// Steffensen's iterations, the step after a cycle's second round t: "y replaces
// x_n and GaBP runs again".  The mean messages of round t move by the cycle's
// scalar step, h <- h^(t) - lam (h^(t) - h^(t-1)) (the precision messages stay),
// and every node record is rebuilt from them: h~ = b + sum h, x = h~ / P~.  With
// stationary precisions these means are exactly y = x^(t) - lam (x^(t) - x^(t-1)).
// Launched after every round; it acts once per even round that has not stopped
// the run (the next round's fused residual then checks the extrapolated iterate).
__global__ void __launch_bounds__(kBlock) k64_steff(Args64 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int t = ctl->round;
  if ((t & 1) || t < 2 || ctl->lam_round == t) return;
  const double lam = ctl->lam;
  const double *__restrict__ b = ctl->b;
  double2 *__restrict__ Mt = a.M0;              // round t (even)
  const double2 *__restrict__ Mp = a.M1;        // round t-1
  NodeRec64 *__restrict__ Nt = a.N0;
  const WarpPos w = warp_pos();
  for (int sl = w.warp; sl < a.ns; sl += w.nwarps) {
    const int i = a.srow[sl * 32 + w.lane];
    const int p0 = a.sp[sl] + w.lane, wd = (a.sp[sl + 1] - a.sp[sl]) >> 5;
    double acch = 0.0;
    for (int j = 0; j < wd; ++j) {
      const int pos = p0 + 32 * j;
      if (a.sci[pos] < 0) break;
      const double ht = Mt[pos].y;
      const double hn = ht - lam * (ht - Mp[pos].y);
      Mt[pos].y = hn;
      acch = __dadd_rn(acch, hn);
    }
    if (i >= 0) {
      const NodeRec64 own = Nt[i];
      const double h = b[i] + acch;
      const double x = h * rcp64(own.P);
      Nt[i] = NodeRec64{own.P, h, x, x};
    }
  }
  // the last block to finish marks round t as extrapolated (every block has passed
  // the guard above by then)
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    ctl->lam_round = t;
    ctl->arrive = 0;
    __threadfence();
  }
}

// Edge-centric round, part 1 (GABP_VARIANT_EDGE): one thread per position computes
// the in-message of its slot from the sender's aggregate minus the reverse message
// (Algorithm 2); padding positions do nothing.
__global__ void __launch_bounds__(kBlock) k64_edge_msg(Args64 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int t = ctl->round + 1;
  const double2 *__restrict__ Min = (t & 1) ? a.M0 : a.M1;
  double2 *__restrict__ Mout = (t & 1) ? a.M1 : a.M0;
  const NodeRec64 *__restrict__ Nin = (t & 1) ? a.N0 : a.N1;
  int bad = 0;
  for (int pos = blockIdx.x * kBlock + threadIdx.x; pos < a.Es; pos += gridDim.x * kBlock) {
    const int k = __ldcs(a.sci + pos);
    if (k < 0) continue;
    const double A = __ldcs(a.sav + pos);
    const double2 rv = __ldcs(Min + __ldcs(a.srev + pos));
    const NodeRec64 nk = Nin[k];
    const double den = nk.P - rv.x;
    bad |= is_zero64(den);
    const double cin = -A * rcp64(den);
    __stcs(Mout + pos, make_double2(__dmul_rn(cin, A), __dmul_rn(cin, nk.h - rv.y)));
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->edge_bad, 1);
}

// Edge-centric round, part 2: row aggregates (the "broadcast" sums of
// Algorithm 2), x^{(t)}, and the residual of x^{(t-1)}.
__global__ void __launch_bounds__(kBlock) k64_edge_agg(Args64 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int t = ctl->round + 1;
  const double *__restrict__ b = ctl->b;
  const double2 *__restrict__ Mnew = (t & 1) ? a.M1 : a.M0;
  const NodeRec64 *__restrict__ Nin = (t & 1) ? a.N0 : a.N1;
  NodeRec64 *__restrict__ Nout = (t & 1) ? a.N1 : a.N0;
  const WarpPos w = warp_pos();
  double rr = 0.0;
  int bad = 0;
  for (int sl = w.warp; sl < a.ns; sl += w.nwarps) {
    const int i = a.srow[sl * 32 + w.lane];
    const int p0 = a.sp[sl] + w.lane, wd = (a.sp[sl + 1] - a.sp[sl]) >> 5;
    double accP = 0.0, acch = 0.0, accr = 0.0;
    for (int j = 0; j < wd; ++j) {
      const int pos = p0 + 32 * j;
      const int k = __ldcs(a.sci + pos);
      if (k < 0) break;
      const double2 m = __ldcs(Mnew + pos);
      accP += m.x;
      acch += m.y;
      accr = fma(__ldcs(a.sav + pos), Nin[k].x, accr);
    }
    if (i >= 0) {
      const double bi = b[i], d = a.ad[i];
      const double P = d + accP, h = bi + acch;
      bad |= is_zero64(P);
      Nout[i] = NodeRec64{P, h, h * rcp64(P), 0.0};
      const double r = bi - fma(d, Nin[i].x, accr);
      rr = fma(r, r, rr);
    }
  }
  double v[2] = {rr, (double)bad}, tot[2];
  const int modes[2] = {0, 0};
  block_sum<2>(v);
  if (last_block_reduce<2>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    const double eb = ctl->edge_bad ? 1.0 : 0.0;
    ctl->edge_bad = 0;
    decide64(ctl, t, tot[0], tot[1] + eb);
  }
}

__global__ void k64_finalize(int n, const NodeRec64 *__restrict__ N, double *__restrict__ x, int aitken) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = aitken ? N[i].pad : N[i].x;
}

// Messages of the returned round in the layout of the input CSR.  M is indexed by
// position c2s[e] of compact slot e (the sliced layout), or by e itself when c2s
// is null.
__global__ void k64_messages(int n, const int *__restrict__ rowptr, const int *__restrict__ dpos,
                             const int *__restrict__ rp, const int *__restrict__ c2s,
                             const double2 *__restrict__ M, double *__restrict__ P, double *__restrict__ hm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = rowptr[i], d = dpos[i], e0 = rp[i], deg = rp[i + 1] - rp[i];
  P[a + d] = 0.0;
  hm[a + d] = 0.0;
  for (int q = 0; q < deg; ++q) {
    int p = a + q + (q >= d ? 1 : 0);
    double2 m = M[c2s ? c2s[e0 + q] : e0 + q];
    P[p] = m.x;
    hm[p] = m.y;
  }
}

// ------------------------------------------------------------------------- sliced layout set-up
// Slot j of row i = srow[q] (q = 32 s + lane) goes to position sp[s] + 32 j + lane.
__global__ void k_sell_fill(int nq, const int *__restrict__ srow, const int *__restrict__ sp,
                            const int *__restrict__ rp, const int *__restrict__ ci, int *__restrict__ c2s,
                            int *__restrict__ sci) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int i = srow[q];
  if (i < 0) return;
  const int p0 = sp[q >> 5] + (q & 31), e0 = rp[i], deg = rp[i + 1] - e0;
  for (int j = 0; j < deg; ++j) {
    c2s[e0 + j] = p0 + 32 * j;
    sci[p0 + 32 * j] = ci[e0 + j];
  }
}

// Reverse positions and values (values again after gabp_set_values).
__global__ void k_sell_rev_vals(int E, const int *__restrict__ c2s, const int *__restrict__ rev,
                                const double *__restrict__ av, int *__restrict__ srev, double *__restrict__ sav,
                                int with_rev) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int pos = c2s[e];
  if (with_rev) srev[pos] = c2s[rev[e]];
  sav[pos] = av[e];
}

__global__ void k64_marginals(int n, const NodeRec64 *__restrict__ N, double *__restrict__ Pi) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Pi[i] = N[i].P;
}

// dL/dA restricted to the pattern and symmetrised: -(lam_i x_j + lam_j x_i)/2
// off the diagonal, -lam_i x_i on it.
__global__ void k_grad_values(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                              const double *__restrict__ lam, const double *__restrict__ x, double *__restrict__ g) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double li = lam[i], xi = x[i];
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
    int j = col[p];
    g[p] = j == i ? -li * xi : -0.5 * (li * x[j] + lam[j] * xi);
  }
}

// ------------------------------------------------------------------------- host side
// The sliced layout of the handle's graph (once per handle; the values again after
// gabp_set_values).  The row order (degree-sorted windows) and the slice offsets are
// computed on the host from the row lengths; the arrays are filled on the device.
// The cluster rounds' shape for a graph of sp.size() - 1 slices, NW warps a CTA: the cluster
// size when both k64_cluster flavours fit on the device, and the shared memory of k64_chip,
// from the slices its CTAs own (slice s to CTA (s mod NW cs) / NW), when that fits too.
template <int NW>
static void cluster_setup(gabp_handle h, const std::vector<int> &sp) {
  const int ns = (int)sp.size() - 1;
  const int cs = std::min(kClusterMax, std::max(1, (ns + NW - 1) / NW));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(32 * NW);
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cs > 8) {
    cudaFuncSetAttribute(k64_cluster<false, NW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k64_cluster<true, NW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  int nc0 = 0, nc1 = 0;  // both flavours must fit (the same cluster serves both)
  if (cudaOccupancyMaxActiveClusters(&nc0, (void *)k64_cluster<false, NW>, &cfg) == cudaSuccess && nc0 > 0 &&
      cudaOccupancyMaxActiveClusters(&nc1, (void *)k64_cluster<true, NW>, &cfg) == cudaSuccess && nc1 > 0) {
    h->clu64 = cs;
    h->clu64_nw = NW;
  }
  cudaGetLastError();
  if (h->clu64 == 0) return;
  const int nw = NW * cs;
  std::vector<int64_t> own_slots(cs, 0), own_rows(cs, 0);
  for (int sl = 0; sl < ns; ++sl) {
    const int o = (sl % nw) / NW;
    own_slots[o] += sp[sl + 1] - sp[sl];
    own_rows[o] += 32;
  }
  const int64_t smax = *std::max_element(own_slots.begin(), own_slots.end());
  const int64_t rmax = *std::max_element(own_rows.begin(), own_rows.end());
  if (smax >= (1 << 24)) return;
  const ChipShape c{(int)smax, (int)rmax};
  const size_t bytes = chip_bytes(c, ns);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  constexpr int kStaticRoom = 1024;  // the kernel's static shared memory (a few hundred bytes) fits below
  if (bytes + kStaticRoom > (size_t)optin) return;
  // The limit is a property of the function, shared by every handle: always the same value, the
  // device's whole opt-in room, so no handle lowers it below another handle's launch size.
  if (cudaFuncSetAttribute(k64_chip<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - kStaticRoom) ==
          cudaSuccess &&
      (cs <= 8 || cudaFuncSetAttribute(k64_chip<NW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess)) {
    cfg.dynamicSmemBytes = bytes;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, (void *)k64_chip<NW>, &cfg) == cudaSuccess && nc > 0) {
      h->chip64_bytes = (int)bytes;
      h->chip64_smax = c.smax;
      h->chip64_rmax = c.rmax;
    }
  }
  cudaGetLastError();
}

static gabp_status ensure_sell64(gabp_handle h) {
  Sell64 &S = h->w64.sl;
  Graph &g = h->g;
  const int n = g.n, E = g.E;
  if (!S.ready) {
    std::vector<int> rp((size_t)n + 1);
    GABP_CUDA(cudaMemcpy(rp.data(), g.rp, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost));
    const int ns = (n + 31) / 32;
    std::vector<int> srow((size_t)ns * 32, -1), sp((size_t)ns + 1, 0);
    std::vector<int> idx;
    for (int w0 = 0; w0 < n; w0 += kSellWindow) {  // a window is a whole number of slices
      const int w1 = std::min(n, w0 + kSellWindow);
      idx.resize(w1 - w0);
      for (int i = w0; i < w1; ++i) idx[i - w0] = i;
      std::stable_sort(idx.begin(), idx.end(),
                       [&](int x, int y) { return rp[x + 1] - rp[x] > rp[y + 1] - rp[y]; });
      std::copy(idx.begin(), idx.end(), srow.begin() + w0);
    }
    int64_t pos = 0;
    for (int sl = 0; sl < ns; ++sl) {
      sp[sl] = (int)pos;
      int wd = 0;
      for (int l = 0; l < 32; ++l) {
        const int i = srow[(size_t)sl * 32 + l];
        if (i >= 0) wd = std::max(wd, rp[i + 1] - rp[i]);
      }
      pos += 32 * (int64_t)wd;
      if (pos >= INT32_MAX) {
        set_last_error("FP64 rounds: the sliced layout does not fit int32 positions");
        return GABP_ERR_INVALID;
      }
    }
    sp[ns] = (int)pos;
    S.ns = ns;
    S.Es = (int)pos;
    const size_t Ea = (size_t)std::max(S.Es, 1), Ec = (size_t)std::max(E, 1);
    GABP_CUDA(cudaMalloc(&S.srow, sizeof(int) * srow.size()));
    GABP_CUDA(cudaMalloc(&S.sp, sizeof(int) * sp.size()));
    GABP_CUDA(cudaMalloc(&S.sci, sizeof(int) * Ea));
    GABP_CUDA(cudaMalloc(&S.srev, sizeof(int) * Ea));
    GABP_CUDA(cudaMalloc(&S.sav, sizeof(double) * Ea));
    GABP_CUDA(cudaMalloc(&S.c2s, sizeof(int) * Ec));
    GABP_CUDA(cudaMemcpyAsync(S.srow, srow.data(), sizeof(int) * srow.size(), cudaMemcpyHostToDevice, h->stream));
    GABP_CUDA(cudaMemcpyAsync(S.sp, sp.data(), sizeof(int) * sp.size(), cudaMemcpyHostToDevice, h->stream));
    GABP_CUDA(cudaMemsetAsync(S.sci, 0xff, sizeof(int) * Ea, h->stream));  // -1: padding
    GABP_CUDA(cudaMemsetAsync(S.srev, 0, sizeof(int) * Ea, h->stream));
    GABP_CUDA(cudaMemsetAsync(S.sav, 0, sizeof(double) * Ea, h->stream));
    const int nq = ns * 32;
    k_sell_fill<<<(nq + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(nq, S.srow, S.sp, g.rp, g.ci, S.c2s, S.sci);
    if (E > 0)
      k_sell_rev_vals<<<(E + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(E, S.c2s, g.rev, g.av, S.srev, S.sav, 1);
    GABP_CUDA(cudaGetLastError());
    GABP_CUDA(cudaStreamSynchronize(h->stream));  // the host vectors are released on return
    S.ready = true;
    S.vals_ok = true;
    h->tuned_L64 = 1;  // one row per lane
    // one cluster of up to 16 CTAs (a slice per warp) for the smallest graphs, its state on chip
    // where it fits
    h->clu64 = h->clu64_nw = 0;
    h->chip64_bytes = h->chip64_smax = h->chip64_rmax = 0;
    if (S.ns <= kClusterMaxSlices) {
      int wmax = 0;  // the widest slice's slots per row
      for (int sl = 0; sl < ns; ++sl) wmax = std::max(wmax, (sp[sl + 1] - sp[sl]) >> 5);
      if (S.ns <= GABP_CLUSTER_NW2_MAX_SLICES) cluster_setup<2>(h, sp);
      else if (S.ns <= 64) cluster_setup<4>(h, sp);
      else if (wmax <= kCluster8MaxWidth) cluster_setup<8>(h, sp);
    }
    // the cooperative launch for small graphs: one block per two slices, all co-resident
    h->coop64 = h->coop64f = 0;
    int coop_attr = 0;
    cudaDeviceGetAttribute(&coop_attr, cudaDevAttrCooperativeLaunch, h->device);
    if (coop_attr && S.ns <= kCoopMaxSlices) {
      const int want = (S.ns * 32 + kCoopThreads - 1) / kCoopThreads;
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k64_coop<false>, kCoopThreads, 0) == cudaSuccess &&
          per_sm > 0)
        h->coop64 = std::min(want, std::min(per_sm * h->num_sms, h->max_blocks));
      per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k64_coop<true>, kCoopThreads, 0) == cudaSuccess &&
          per_sm > 0)
        h->coop64f = std::min(want, std::min(per_sm * h->num_sms, h->max_blocks));
      cudaGetLastError();
    }
  } else if (!S.vals_ok) {
    if (E > 0)
      k_sell_rev_vals<<<(E + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(E, S.c2s, g.rev, g.av, S.srev, S.sav, 0);
    GABP_CUDA(cudaGetLastError());
    S.vals_ok = true;
  }
  return GABP_OK;
}

gabp_status ensure_w64(gabp_handle h) {
  gabp_status s = ensure_sell64(h);
  if (s != GABP_OK) return s;
  Work64 &w = h->w64;
  if (w.M[0]) return GABP_OK;
  size_t Es = (size_t)std::max(w.sl.Es, 1), n = (size_t)h->g.n;
  GABP_CUDA(cudaMalloc(&w.M[0], sizeof(double2) * Es));
  GABP_CUDA(cudaMalloc(&w.M[1], sizeof(double2) * Es));
  GABP_CUDA(cudaMalloc(&w.N[0], sizeof(NodeRec64) * n));
  GABP_CUDA(cudaMalloc(&w.N[1], sizeof(NodeRec64) * n));
  return GABP_OK;
}

void free_w64(gabp_handle h) {
  Work64 &w = h->w64;
  cudaFree(w.M[0]); cudaFree(w.M[1]); cudaFree(w.N[0]); cudaFree(w.N[1]); cudaFree(w.bar); cudaFree(w.C);
  Sell64 &S = w.sl;
  cudaFree(S.srow); cudaFree(S.sp); cudaFree(S.sci); cudaFree(S.srev); cudaFree(S.sav); cudaFree(S.c2s);
  w = Work64{};
}

static Args64 args64(gabp_handle h) {
  Args64 a;
  const Sell64 &S = h->w64.sl;
  a.n = h->g.n;
  a.ns = S.ns;
  a.Es = S.Es;
  a.srow = S.srow;
  a.sp = S.sp;
  a.sci = S.sci;
  a.srev = S.srev;
  a.sav = S.sav;
  a.ad = h->g.ad;
  a.M0 = h->w64.M[0];
  a.M1 = h->w64.M[1];
  a.N0 = h->w64.N[0];
  a.N1 = h->w64.N[1];
  a.ctl = h->ctl;
  a.partials = h->partials;
  a.C = h->w64.C;
  a.freeze = h->opt.freeze_precisions && h->opt.variant == GABP_VARIANT_NODE && h->opt.accel == ACC_NONE &&
             h->w64.C != nullptr;
  // long rows and too few slices to give every SM eight warps: a warp per row instead
  a.wide = !a.freeze && h->opt.variant == GABP_VARIANT_NODE && h->opt.accel == ACC_NONE && S.ns > 0 &&
           (double)S.Es >= 64.0 * 32.0 * S.ns && S.ns < 8 * h->num_sms;
  return a;
}

template <typename K>
static int slice_grid(gabp_handle h, K kernel) {
  return blocks_for(h->w64.sl.ns, kBlock / 32, resident_grid(h->num_sms, kernel));
}

static void launch_round(gabp_handle h, const Args64 &a) {
  if (h->opt.variant == GABP_VARIANT_EDGE) {
    const int eb = blocks_for(a.Es, kBlock, resident_grid(h->num_sms, k64_edge_msg));
    k64_edge_msg<<<eb, kBlock, 0, h->stream>>>(a);
    k64_edge_agg<<<slice_grid(h, k64_edge_agg), kBlock, 0, h->stream>>>(a);
  } else if (h->opt.accel == ACC_AITKEN) {
    k64_node<ACC_AITKEN><<<slice_grid(h, k64_node<ACC_AITKEN>), kBlock, 0, h->stream>>>(a);
  } else if (h->opt.accel == ACC_STEFFENSEN) {
    k64_node<ACC_STEFFENSEN><<<slice_grid(h, k64_node<ACC_STEFFENSEN>), kBlock, 0, h->stream>>>(a);
    k64_steff<<<slice_grid(h, k64_steff), kBlock, 0, h->stream>>>(a);
  } else if (a.wide) {
    k64_wide<<<resident_grid(h->num_sms, k64_wide), kBlock, 0, h->stream>>>(a);
  } else if (a.freeze) {
    k64_frz<3><<<slice_grid(h, k64_frz<3>), kBlock, 0, h->stream>>>(a);
    k64_frz<2><<<slice_grid(h, k64_frz<2>), kBlock, 0, h->stream>>>(a);
    k64_frz<1><<<slice_grid(h, k64_frz<1>), kBlock, 0, h->stream>>>(a);
  } else {
    k64_node<ACC_NONE><<<slice_grid(h, k64_node<ACC_NONE>), kBlock, 0, h->stream>>>(a);
  }
}

// K rounds as one CUDA graph (the round index lives in device memory, so the
// same graph serves every replay and every solve on this handle).
static gabp_status get_graph64(gabp_handle h, cudaGraphExec_t *out) {
  const int K = h->opt.check_every;
  const int key = (h->opt.variant << 12) ^ (h->opt.accel << 24) ^ (h->opt.freeze_precisions << 28) ^ K;
  if (h->g64 && h->g64_key == key) {
    *out = h->g64;
    return GABP_OK;
  }
  if (h->g64) cudaGraphExecDestroy(h->g64);
  h->g64 = nullptr;
  Args64 a = args64(h);
  cudaGraph_t graph;
  GABP_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < K; ++k) launch_round(h, a);
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (e != cudaSuccess) return cuda_fail(e, "capture FP64 rounds");
  e = cudaGraphInstantiate(&h->g64, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "instantiate FP64 rounds");
  h->g64_key = key;
  *out = h->g64;
  return GABP_OK;
}

gabp_status solve64(gabp_handle h, const double *b, double *x, double tol, int max_iter, int *iters,
                    double *relres) {
  NvtxRange nvtx_("gabp fp64 rounds");
  gabp_status s = ensure_w64(h);
  if (s != GABP_OK) return s;
  Graph &g = h->g;
  const size_t Es = (size_t)std::max(h->w64.sl.Es, 1);
  // warm start: the messages of the previous FP64 solve (or imported ones) as round 0
  const bool warm = h->opt.warm_start && h->w64.valid;
  if (warm && (h->w64.result_round & 1))
    GABP_CUDA(cudaMemcpyAsync(h->w64.M[0], h->w64.M[1], sizeof(double2) * Es, cudaMemcpyDeviceToDevice,
                              h->stream));
  h->w64.valid = false;
  if (h->opt.freeze_precisions && !h->w64.C)  // the frozen coefficients' store
    GABP_CUDA(cudaMalloc(&h->w64.C, sizeof(double) * Es));
  Args64 a = args64(h);
  // round-0 state (Algorithm 1 step 1): control block pointed at b, zero messages
  auto init = [&]() -> gabp_status {
    GABP_CUDA(cudaMemsetAsync(h->ctl, 0, sizeof(DevCtl), h->stream));
    const double *bptr = b;
    GABP_CUDA(cudaMemcpyAsync(&h->ctl->b, &bptr, sizeof(bptr), cudaMemcpyHostToDevice, h->stream));
    if (h->opt.history > 0) {  // per-round residual history (options.history entries)
      if (h->hist_alloc < h->opt.history) {
        cudaFree(h->hist);
        h->hist = nullptr;
        h->hist_alloc = 0;
        GABP_CUDA(cudaMalloc(&h->hist, sizeof(double) * (size_t)h->opt.history));
        h->hist_alloc = h->opt.history;
      }
      double *hp = h->hist;
      const int cap = h->opt.history;
      GABP_CUDA(cudaMemcpyAsync(&h->ctl->hist, &hp, sizeof(hp), cudaMemcpyHostToDevice, h->stream));
      GABP_CUDA(cudaMemcpyAsync(&h->ctl->hist_cap, &cap, sizeof(cap), cudaMemcpyHostToDevice, h->stream));
    }
    if (!warm) GABP_CUDA(cudaMemsetAsync(h->w64.M[0], 0, sizeof(double2) * Es, h->stream));
    k64_init<<<blocks_for(a.ns, kBlock / 32, h->max_blocks), kBlock, 0, h->stream>>>(a, tol, max_iter, warm ? 1 : 0);
    GABP_CUDA(cudaGetLastError());
    GABP_CUDA(cudaStreamSynchronize(h->stream));  // also retires the pageable copy of bptr
    return GABP_OK;
  };
  if ((s = init()) != GABP_OK) return s;

  // small and medium graphs: every round in one cooperative launch
  const int coop_grid = a.freeze ? h->coop64f : h->coop64;
  const bool clus = !a.wide && h->w64.sl.ns <= kClusterMaxSlices && h->opt.variant == GABP_VARIANT_NODE &&
                    h->opt.accel == ACC_NONE && h->clu64 > 0;
  const bool coop = !clus && !a.wide && h->w64.sl.ns <= kCoopMaxSlices && h->opt.variant == GABP_VARIANT_NODE &&
                    h->opt.accel == ACC_NONE && coop_grid > 0;
  const bool use_graph = !coop && !clus && h->stream != nullptr && h->opt.graphs;
  cudaGraphExec_t ge = nullptr;
  if (use_graph) {
    s = get_graph64(h, &ge);
    if (s != GABP_OK) return s;
  }
  const int K = h->opt.check_every;
  const int64_t max_batches = (int64_t)(max_iter + 2) / K + 3;
  bool done = false;
  if ((s = read_ctl(h)) != GABP_OK) return s;
  done = h->ctl_host->done;
  const int per_round =
      a.freeze ? 3 : h->opt.variant == GABP_VARIANT_EDGE || h->opt.accel == ACC_STEFFENSEN ? 2 : 1;
  h->prof.launches += 1;  // k64_init
  int prev_round = 0;
  if (!done && clus) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = h->clu64;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(h->clu64);
    cfg.blockDim = dim3(32 * h->clu64_nw);
    cfg.stream = h->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int max_rounds = max_iter + 2;
    // plain rounds with the state on chip where it fits (the same values: same slices, lanes and sums)
    const bool chip = !a.freeze && h->chip64_bytes > 0;
    if (chip) cfg.dynamicSmemBytes = h->chip64_bytes;
    prof_begin(h);
    const ChipShape cs{h->chip64_smax, h->chip64_rmax};
    cudaError_t le;
    if (h->clu64_nw == 2)
      le = chip ? cudaLaunchKernelEx(&cfg, k64_chip<2>, a, cs, max_rounds)
           : a.freeze ? cudaLaunchKernelEx(&cfg, k64_cluster<true, 2>, a, max_rounds)
                      : cudaLaunchKernelEx(&cfg, k64_cluster<false, 2>, a, max_rounds);
    else if (h->clu64_nw == 4)
      le = chip ? cudaLaunchKernelEx(&cfg, k64_chip<4>, a, cs, max_rounds)
           : a.freeze ? cudaLaunchKernelEx(&cfg, k64_cluster<true, 4>, a, max_rounds)
                      : cudaLaunchKernelEx(&cfg, k64_cluster<false, 4>, a, max_rounds);
    else
      le = chip ? cudaLaunchKernelEx(&cfg, k64_chip<8>, a, cs, max_rounds)
           : a.freeze ? cudaLaunchKernelEx(&cfg, k64_cluster<true, 8>, a, max_rounds)
                      : cudaLaunchKernelEx(&cfg, k64_cluster<false, 8>, a, max_rounds);
    if (le != cudaSuccess) return cuda_fail(le, "FP64 cluster rounds");
    prof_end(h);
    h->prof.launches += 1;
    if ((s = read_ctl(h)) != GABP_OK) return s;
    prof_collect(h, PH_FP64, h->ctl_host->round);
    done = h->ctl_host->done;
  }
  if (!done && coop) {
    Work64 &w = h->w64;
    if (!w.bar) GABP_CUDA(cudaMalloc(&w.bar, 16));  // [0] arrivals, [1] generation, [2] error flag
    GABP_CUDA(cudaMemsetAsync(w.bar, 0, 16, h->stream));
    unsigned *bar = w.bar;
    int *err = reinterpret_cast<int *>(w.bar + 2);
    int max_rounds = max_iter + 2;
    void *args[] = {(void *)&a, (void *)&bar, (void *)&err, (void *)&max_rounds};
    prof_begin(h);
    cudaError_t le = cudaLaunchCooperativeKernel(a.freeze ? (void *)k64_coop<true> : (void *)k64_coop<false>,
                                                 dim3(coop_grid), dim3(kCoopThreads), args, 0, h->stream);
    if (le != cudaSuccess) return cuda_fail(le, "FP64 cooperative rounds");
    prof_end(h);
    h->prof.launches += 1;
    int herr = 0;
    GABP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    if ((s = read_ctl(h)) != GABP_OK) return s;
    prof_collect(h, PH_FP64, h->ctl_host->round);
    if (herr) {
      set_last_error("FP64 cooperative rounds: a grid barrier gave up");
      return GABP_TIMEOUT;
    }
    done = h->ctl_host->done;
  }
  for (int64_t batch = 0; !done && !coop && !clus && batch < max_batches; ++batch) {
    prof_begin(h);
    if (use_graph) {
      GABP_CUDA(cudaGraphLaunch(ge, h->stream));
    } else {
      for (int k = 0; k < K; ++k) launch_round(h, a);
      GABP_CUDA(cudaGetLastError());
    }
    prof_end(h);
    h->prof.launches += (int64_t)K * per_round;
    if ((s = read_ctl(h)) != GABP_OK) return s;
    prof_collect(h, PH_FP64, h->ctl_host->round - prev_round);
    prev_round = h->ctl_host->round;
    done = h->ctl_host->done;
  }
  if (!done) {
    set_last_error("solve64: control loop ended without a decision");
    return GABP_ERR_CUDA;
  }
  const DevCtl c = *h->ctl_host;
  h->w64.result_round = c.result_round;
  h->w64.valid = true;
  h->hist_len = h->opt.history > 0 ? c.hist_len : 0;
  h->hist_bb = c.bb;
  h->stats.rounds = c.round;
  h->stats.edge_updates = -1;
  h->stats.refine_steps = 0;
  h->stats.freeze_round = a.freeze ? c.fround : 0;
  h->stats.freeze_checks = a.freeze ? c.fchecks : 0;
  if (warm && c.bb == 0.0) {  // b = 0: x = 0 (the warm round-0 records hold the old messages' mean)
    GABP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * g.n, h->stream));
  } else {
    k64_finalize<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, h->w64.N[c.result_round & 1], x,
                                                                       h->opt.accel == ACC_AITKEN);
    h->prof.launches += 1;
  }
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  if (iters) *iters = c.iters;
  if (relres) *relres = c.bb > 0.0 ? sqrt(c.rr / c.bb) : 0.0;
  return (gabp_status)c.status;
}

gabp_status messages64(gabp_handle h, double *P, double *hm) {
  if (!h->w64.valid) return GABP_ERR_INVALID;
  Graph &g = h->g;
  k64_messages<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(
      g.n, g.rowptr, g.dpos, g.rp, h->w64.sl.c2s, h->w64.M[h->w64.result_round & 1], P, hm);
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return GABP_OK;
}

// Inverse of k64_messages: input-layout messages into the sliced positions.
__global__ void k64_load_messages(int n, const int *__restrict__ rowptr, const int *__restrict__ dpos,
                                  const int *__restrict__ rp, const int *__restrict__ c2s,
                                  const double *__restrict__ P, const double *__restrict__ hm,
                                  double2 *__restrict__ M) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = rowptr[i], d = dpos[i], e0 = rp[i], deg = rp[i + 1] - rp[i];
  for (int q = 0; q < deg; ++q) {
    int p = a + q + (q >= d ? 1 : 0);
    M[c2s[e0 + q]] = make_double2(P[p], hm[p]);
  }
}

gabp_status load_messages64(gabp_handle h, const double *P, const double *hm) {
  gabp_status s = ensure_w64(h);
  if (s != GABP_OK) return s;
  Graph &g = h->g;
  k64_load_messages<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, g.rowptr, g.dpos, g.rp,
                                                                           h->w64.sl.c2s, P, hm, h->w64.M[0]);
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  h->w64.result_round = 0;
  h->w64.valid = true;
  return GABP_OK;
}

gabp_status messages64_from(gabp_handle h, const double2 *M, double *P, double *hm) {
  Graph &g = h->g;
  k64_messages<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, g.rowptr, g.dpos, g.rp, nullptr, M, P,
                                                                       hm);
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return GABP_OK;
}

gabp_status marginals(gabp_handle h, double *Pi) {
  if (!h->w64.valid) return GABP_ERR_INVALID;
  Graph &g = h->g;
  k64_marginals<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, h->w64.N[h->w64.result_round & 1], Pi);
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return GABP_OK;
}

gabp_status grad_values(gabp_handle h, const double *lam, const double *x, double *gv) {
  Graph &g = h->g;
  k_grad_values<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, g.rowptr, g.col, lam, x, gv);
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return GABP_OK;
}

}  // namespace gabp
