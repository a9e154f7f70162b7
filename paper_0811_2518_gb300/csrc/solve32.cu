// solve32.cu -- FP32 messages + FP64 iterative refinement, and the convergence fix.
//
// The precision messages do not depend on b (eq_prec, eq_prec_message: P_ij =
// -A_ij^2 / P_{i\j}), so they are iterated once per matrix, then frozen.  With
// P frozen, the information-form mean message is linear in the cavity:
//   h_ij = c_ij (h~_i - h_ji),   c_ij = -A_ij / (P~_i - P_ji)       (Algorithm 2),
// and x_i = h~_i / P~_i.  These iterations run in FP32; the only FP64 steps are
// the outer residual r = b - A x and the update x <- x + d, where d is the FP32
// GaBP solution of A d = r.  With a diagonal loading Gamma the inner solves run
// on A + Gamma and the same outer loop is the paper's convergence fix
//   x^(t+1) = x^(t) + (A + Gamma)^{-1} (b - A x^(t)) = (A + Gamma)^{-1}(b + Gamma x^(t))
// (Chapter "Fixing convergence of GaBP", eq:iterative_method).
//
// Recompute form.  Slot e of row i (sender k) keeps its own in-message in one of
// two chains (even / odd rounds).  Round t needs the reverse message i -> k of
// round t-1, which row i itself can recompute from what it held at round t-2:
//   h_{i->k}^{(t-1)} = c_out (h~_i^{(t-2)} - h_{k->i}^{(t-2)}),
//   h_{k->i}^{(t)}   = c_in  (h~_k^{(t-1)} - h_{i->k}^{(t-1)}),
// with c_in = c_ki and c_out = c_ik stored side by side in slot e.  The same
// holds for the precision messages.  Every edge array is then read and written
// in place, coalesced, with no gather or scatter through rev[]; only the node
// values h~_k^{(t-1)} are gathered (they stay in L2).  In exact arithmetic this
// is the synchronous schedule of Algorithm 2; in FP32 it rounds the same way as
// computing h_{i->k}^{(t-1)} once and storing it.
#include "gabp_internal.cuh"
#include "devutil.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

namespace gabp {

constexpr int kPrecMaxRounds = 300;  // cap of the FP32 precision phase
constexpr int kUnroll32 = 4;         // default slots per lane whose loads are issued together

// Round-kernel shapes the autotuner chooses from: (lanes per row L, slots per
// lane whose loads are issued together U), packed as L | U << 8.
constexpr int shape_code(int L, int U) { return L | (U << 8); }
constexpr int kShapes[] = {shape_code(1, 4), shape_code(2, 4), shape_code(4, 4), shape_code(8, 4),
                           shape_code(1, 8), shape_code(2, 8), shape_code(4, 8),
                           shape_code(2, 2), shape_code(4, 2), shape_code(8, 2),
                           shape_code(16, 1), shape_code(16, 2)};
template <int V> using IC = std::integral_constant<int, V>;

// The shape a pinned (options.lanes, options.unroll) pair selects, or 0 if the
// library has no such kernel.
int pinned_shape32(int lanes, int unroll) {
  const int L = lanes > 16 ? 16 : lanes;
  const int U = unroll ? unroll : (L >= 16 ? 1 : kUnroll32);
  for (int sc : kShapes)
    if (sc == shape_code(L, U)) return sc;
  return 0;
}

// f(IC<L>, IC<U>) for a shape code (unknown codes map to (4, 4)).
template <typename F>
void with_shape(int code, F &&f) {
  switch (code) {
    case shape_code(1, 4): f(IC<1>{}, IC<4>{}); break;
    case shape_code(2, 4): f(IC<2>{}, IC<4>{}); break;
    case shape_code(8, 4): f(IC<8>{}, IC<4>{}); break;
    case shape_code(1, 8): f(IC<1>{}, IC<8>{}); break;
    case shape_code(2, 8): f(IC<2>{}, IC<8>{}); break;
    case shape_code(4, 8): f(IC<4>{}, IC<8>{}); break;
    case shape_code(2, 2): f(IC<2>{}, IC<2>{}); break;
    case shape_code(4, 2): f(IC<4>{}, IC<2>{}); break;
    case shape_code(8, 2): f(IC<8>{}, IC<2>{}); break;
    case shape_code(16, 1): f(IC<16>{}, IC<1>{}); break;
    case shape_code(16, 2): f(IC<16>{}, IC<2>{}); break;
    default: f(IC<4>{}, IC<4>{}); break;
  }
}

struct Args32 {
  int n;
  int dense;  // complete pattern (a dense matrix): k32_mean derives the sender from the slot
  const int *__restrict__ rp;
  const int *__restrict__ ci;
  const float *__restrict__ av;
  const float *__restrict__ ad;   // diagonal of the matrix the inner solves run on (A + Gamma)
  float *MP0, *MP1;               // precision chains
  float *NP0, *NP1, *NP2;         // P~ ring
  float2 *CF;                     // {c_in, c_out}
  float *invP;
  float *H0, *H1;                 // mean chains
  float *NH0, *NH1, *NH2;         // h~ ring
  const float *rhs;               // FP32 right-hand side of the inner solve
  float2 *NQ0, *NQ1, *NQ2;        // {P~, h~} ring of the joint rounds
  DevCtl *ctl;
  double *partials;
  cudaGraphConditionalHandle cond;  // while-node condition cleared when the run is decided
  int use_cond;                     // (only inside the device-loop graph)
};

__device__ __forceinline__ float *ring3(float *a, float *b, float *c, int t) {
  int m = t % 3;
  return m == 0 ? a : (m == 1 ? b : c);
}
__device__ __forceinline__ float2 *ring3(float2 *a, float2 *b, float2 *c, int t) {
  int m = t % 3;
  return m == 0 ? a : (m == 1 ? b : c);
}

// ---------------------------------------------------------------------------- precision phase
// Round t of the precision-only iteration (eq_prec + eq_prec_message, Algorithm 2),
// recompute form.  The run stops once every message has |P^(t) - P^(t-1)| <=
// 2^-s |P^(t)| (s = options.prec_stop_log2, default 16; kept in ctl->tol2bb)
// in two consecutive rounds, on a zero cavity, or at max_iter; a non-finite
// message after round 1 stops it as diverged.  The reciprocals use the fast
// FP32 division (__fdividef, about 2 ulp): the FP32 precision state only has to
// be FP32-accurate, the FP64 refinement absorbs what the frozen coefficients are
// off by (|divisor| >= 2^126 would give 0; such precisions are outside FP32's use).
// FP32 rounding keeps some messages moving by a few ulp forever, so an exact
// stationary point is not waited for: the outer FP64 refinement absorbs what
// the frozen coefficients are off by.
template <int L, int U>
__global__ void __launch_bounds__(kBlock) k32_prec(Args32 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int t = ctl->round + 1;
  float *__restrict__ Mc = (t & 1) ? a.MP1 : a.MP0;        // holds t-2, becomes t
  const float *__restrict__ Mo = (t & 1) ? a.MP0 : a.MP1;  // holds t-1
  const float *__restrict__ Pm1 = ring3(a.NP0, a.NP1, a.NP2, t + 2);
  const float *__restrict__ Pm2 = ring3(a.NP0, a.NP1, a.NP2, t + 1);
  float *__restrict__ Pt = ring3(a.NP0, a.NP1, a.NP2, t);
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  const float thr = (float)ctl->tol2bb;  // 2^-prec_stop_log2
  int bad = 0, moving = 0, nonfinite = 0;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int i = base + sw;
    float acc = 0.f;
    if (i < a.n) {
      const float Pi2 = t >= 2 ? Pm2[i] : 0.f;
      const int e1 = a.rp[i + 1];
      for (int eb = a.rp[i] + sl; eb < e1; eb += L * U) {
        // all loads of U slots first (memory-level parallelism), then the gathers
        int k[U];
        float A[U], Ps[U], Pp[U], Pk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = eb + u * L;
          if (e < e1) { k[u] = __ldcs(a.ci + e); A[u] = __ldcs(a.av + e); Ps[u] = __ldcs(Mc + e); Pp[u] = __ldcs(Mo + e); }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (eb + u * L < e1) Pk[u] = Pm1[k[u]];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = eb + u * L;
          if (e < e1) {
            const float A2 = A[u] * A[u];
            float Pout = 0.f;
            if (t >= 2) {
              const float d1 = Pi2 - Ps[u];
              bad |= (d1 == 0.f);
              Pout = -A2 * __fdividef(1.f, d1);
            }
            const float d2 = Pk[u] - Pout;
            bad |= (d2 == 0.f);
            const float Pn = -A2 * __fdividef(1.f, d2);
            __stcs(Mc + e, Pn);
            acc += Pn;
            moving |= !(fabsf(Pn - Pp[u]) <= thr * fabsf(Pn));  // a NaN counts as moving
            nonfinite |= !isfinite(Pn);
          }
        }
      }
    }
    acc = sub_sum<L>(acc);
    if (i < a.n && sl == 0) {
      const float P = a.ad[i] + acc;
      bad |= (P == 0.f);
      Pt[i] = P;
    }
  }
  double v[3] = {(double)bad, (double)moving, (double)nonfinite}, tot[3];
  block_sum<3>(v);
  const int modes[3] = {0, 0, 0};
  if (last_block_reduce<3>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    ctl->round = t;
    ctl->maxrel = tot[1];                      // messages that moved by more than 2^-s
    ctl->stable = tot[1] == 0.0 ? ctl->stable + 1 : 0;
    if (ctl->no_stop) {
      // autotuning run: no decision
    } else if (tot[0] > 0.0) {
      ctl->status = GABP_BREAKDOWN; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (tot[2] > 0.0 && t > 1) {
      ctl->status = GABP_DIVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (ctl->stable >= 2) {
      ctl->status = GABP_OK; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (t >= ctl->max_iter) {
      ctl->status = GABP_NOT_CONVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    }
    ctl->arrive = 0;
    __threadfence();
  }
}

// ---------------------------------------------------------------------------- joint rounds
// Round t of the full FP32 iteration (Algorithm 2: eq_prec_message and
// eq_mean_message for every directed edge, in information form), recompute form
// for both messages.  Slot e = (i, k) keeps the in-messages P_ki, h_ki; the
// reverse messages of round t-1 are recomputed from row i's own round t-2 state:
//   P_ik = -A^2 / (P~_i - P_ki),  h_ik = -A (h~_i - h_ki) / (P~_i - P_ki),
// then  P_ki^t = -A^2 / (P~_k - P_ik),  h_ki^t = -A (h~_k - h_ik) / (P~_k - P_ik)
// with the sender's round t-1 aggregates {P~_k, h~_k} fetched as ONE 8-byte
// gather.  The node aggregates go to the {P~, h~} ring and to the P~ and h~ rings
// the precision-only and frozen-coefficient kernels read, so the run can freeze
// the coefficients at any round T and continue with k32_mean from round T + 1.
// Stop rule: the precision phase's (relative change <= 2^-s in two consecutive
// rounds, zero cavity, max_iter).
template <int L, int U>
__global__ void __launch_bounds__(kBlock, 4) k32_joint(Args32 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int t = ctl->round + 1;
  float *__restrict__ Mc = (t & 1) ? a.MP1 : a.MP0;        // P chain: holds t-2, becomes t
  const float *__restrict__ Mo = (t & 1) ? a.MP0 : a.MP1;  // P at t-1
  float *__restrict__ Hc = (t & 1) ? a.H1 : a.H0;          // h chain: holds t-2, becomes t
  const float2 *__restrict__ Qm1 = ring3(a.NQ0, a.NQ1, a.NQ2, t + 2);
  const float2 *__restrict__ Qm2 = ring3(a.NQ0, a.NQ1, a.NQ2, t + 1);
  float2 *__restrict__ Qt = ring3(a.NQ0, a.NQ1, a.NQ2, t);
  float *__restrict__ Pt = ring3(a.NP0, a.NP1, a.NP2, t);
  float *__restrict__ Ht = ring3(a.NH0, a.NH1, a.NH2, t);
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  const float thr = (float)ctl->tol2bb;  // 2^-prec_stop_log2
  int bad = 0, moving = 0, nonfinite = 0;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int i = base + sw;
    float accP = 0.f, accH = 0.f, ad_i = 0.f, rhs_i = 0.f;
    if (i < a.n) {
      const float2 q2 = t >= 2 ? Qm2[i] : make_float2(0.f, 0.f);
      ad_i = a.ad[i];  // requested before the slots (latency overlap)
      rhs_i = a.rhs[i];
      const int e1 = a.rp[i + 1];
      for (int eb = a.rp[i] + sl; eb < e1; eb += L * U) {
        int k[U];
        float A[U], Ps[U], Pp[U], hs[U];
        float2 qk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = eb + u * L;
          if (e < e1) {
            k[u] = __ldcs(a.ci + e); A[u] = __ldcs(a.av + e);
            Ps[u] = __ldcs(Mc + e); Pp[u] = __ldcs(Mo + e); hs[u] = __ldcs(Hc + e);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (eb + u * L < e1) qk[u] = __ldcg(Qm1 + k[u]);  // random gather, L2 only
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = eb + u * L;
          if (e < e1) {
            float Pout = 0.f, hout = 0.f;
            if (t >= 2) {  // message i -> k of round t-1
              const float d1 = q2.x - Ps[u];
              bad |= (d1 == 0.f);
              const float r1 = __fdividef(1.f, d1);
              Pout = -A[u] * A[u] * r1;
              hout = -A[u] * (q2.y - hs[u]) * r1;
            }
            const float d2 = qk[u].x - Pout;  // message k -> i of round t
            bad |= (d2 == 0.f);
            const float r2 = __fdividef(1.f, d2);
            const float Pn = -A[u] * A[u] * r2;
            const float hn = -A[u] * (qk[u].y - hout) * r2;
            __stcs(Mc + e, Pn);
            __stcs(Hc + e, hn);
            accP += Pn;
            accH += hn;
            moving |= !(fabsf(Pn - Pp[u]) <= thr * fabsf(Pn));  // a NaN counts as moving
            nonfinite |= !isfinite(Pn);
          }
        }
      }
    }
    accP = sub_sum<L>(accP);
    accH = sub_sum<L>(accH);
    if (i < a.n && sl == 0) {
      const float P = ad_i + accP, hh = rhs_i + accH;
      bad |= (P == 0.f);
      Qt[i] = make_float2(P, hh);
      Pt[i] = P;
      Ht[i] = hh;
    }
  }
  double v[3] = {(double)bad, (double)moving, (double)nonfinite}, tot[3];
  block_sum<3>(v);
  const int modes[3] = {0, 0, 0};
  if (last_block_reduce<3>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    ctl->round = t;
    ctl->maxrel = tot[1];                      // messages that moved by more than 2^-s
    ctl->stable = tot[1] == 0.0 ? ctl->stable + 1 : 0;
    if (ctl->no_stop) {
      // autotuning run: no decision
    } else if (tot[0] > 0.0) {
      ctl->status = GABP_BREAKDOWN; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (tot[2] > 0.0 && t > 1) {
      ctl->status = GABP_DIVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (ctl->stable >= 2) {
      ctl->status = GABP_OK; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (t >= ctl->max_iter) {
      ctl->status = GABP_NOT_CONVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    }
    if (a.use_cond && ctl->done) cudaGraphSetConditional(a.cond, 0);
    ctl->arrive = 0;
    __threadfence();
  }
}

// round-0 state of the joint rounds: zero messages, {P~, h~} = {A_ii (+ Gamma_ii), r}
__global__ void k32_joint_init(int n, const float *__restrict__ ad, const float *__restrict__ rhs, float2 *nq0,
                               float *np0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    nq0[i] = make_float2(ad[i], rhs[i]);
    np0[i] = ad[i];
  }
}

// Freeze: c_out = c_ik = -A / (P~_i - P_ki), P_ik = c_out A, c_in = c_ki = -A / (P~_k - P_ik),
// 1/P~_i.  Uses round T's precision state.
template <int L>
__global__ void __launch_bounds__(kBlock) k32_coef(Args32 a, int T) {
  const float *__restrict__ Ms = (T & 1) ? a.MP1 : a.MP0;
  const float *__restrict__ PT = ring3(a.NP0, a.NP1, a.NP2, T);
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int i = base + sw;
    if (i >= a.n) continue;
    const float Pi = PT[i];
    for (int e = a.rp[i] + sl; e < a.rp[i + 1]; e += L) {
      const int k = a.ci[e];
      const float A = a.av[e];
      const float cout = -A / (Pi - Ms[e]);
      const float Pout = cout * A;
      const float cin = -A / (PT[k] - Pout);
      a.CF[e] = make_float2(cin, cout);
    }
    if (sl == 0) a.invP[i] = 1.f / Pi;
  }
}

// ---------------------------------------------------------------------------- mean phase, one RHS
// Round t of the frozen-precision mean iteration (recompute form).  The inner
// solve stops when ||x^(t) - x^(t-1)|| <= inner_tol ||x^(t)|| (node-local
// quantities, no extra edge traffic) or at max_iter.
template <int L, int U, bool DENSE = false>
__global__ void __launch_bounds__(kBlock) k32_mean(Args32 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int t = ctl->round + 1;
  float *__restrict__ Hc = (t & 1) ? a.H1 : a.H0;  // holds t-2, becomes t
  const float *__restrict__ Hm1 = ring3(a.NH0, a.NH1, a.NH2, t + 2);
  const float *__restrict__ Hm2 = ring3(a.NH0, a.NH1, a.NH2, t + 1);
  float *__restrict__ Ht = ring3(a.NH0, a.NH1, a.NH2, t);
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  float dxx = 0.f, xx = 0.f;  // per-thread partial sums stay in FP32 (the FP64 pipe is narrow)
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int i = base + sw;
    float acc = 0.f, rhs_i = 0.f, ip = 0.f, hprev = 0.f;
    if (i < a.n) {
      // the row's own values are requested before its slots, so that their latency overlaps the slot loads
      const float hi2 = t >= 2 ? Hm2[i] : 0.f;
      rhs_i = a.rhs[i];
      ip = a.invP[i];
      hprev = Hm1[i];
      const int e0 = a.rp[i], e1 = a.rp[i + 1];
      for (int eb = e0 + sl; eb < e1; eb += L * U) {
        int k[U];
        float2 cf[U];
        float hs[U], hk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = eb + u * L;
          if (e < e1) {
            // a complete pattern: slot p of row i holds column p + (p >= i), no column stream
            k[u] = DENSE ? (e - e0) + (e - e0 >= i) : __ldcs(a.ci + e);
            cf[u] = __ldcs(a.CF + e);
            hs[u] = __ldcs(Hc + e);
          }
        }
        // random gathers bypass L1 (no reuse there), which keeps L1 for the slot streams' sectors; a
        // complete pattern reads the aggregates in column order, the same vector in every row: L1
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (eb + u * L < e1) hk[u] = DENSE ? __ldg(Hm1 + k[u]) : __ldcg(Hm1 + k[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = eb + u * L;
          if (e < e1) {
            const float hout = t >= 2 ? cf[u].y * (hi2 - hs[u]) : 0.f;  // message i -> k at t-1
            const float hn = cf[u].x * (hk[u] - hout);                  // message k -> i at t
            __stcs(Hc + e, hn);
            acc += hn;
          }
        }
      }
    }
    acc = sub_sum<L>(acc);
    if (i < a.n && sl == 0) {
      const float hnew = rhs_i + acc;
      Ht[i] = hnew;
      const float x = hnew * ip, dx = (hnew - hprev) * ip;
      dxx = fmaf(dx, dx, dxx);
      xx = fmaf(x, x, xx);
    }
  }
  double v[2] = {(double)dxx, (double)xx}, tot[2];
  const int modes[2] = {0, 0};
  block_sum<2>(v);
  if (last_block_reduce<2>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    ctl->round = t;
    ctl->rr = tot[0];
    ctl->xx = tot[1];
    if (ctl->no_stop) {
      // autotuning run: no decision
    } else if (!isfinite(tot[0]) || !isfinite(tot[1])) {
      ctl->status = GABP_DIVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (t >= 2 && tot[0] <= ctl->tol2bb * tot[1]) {
      ctl->status = GABP_OK; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (t >= ctl->max_iter) {
      ctl->status = GABP_NOT_CONVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    }
    if (a.use_cond && ctl->done) cudaGraphSetConditional(a.cond, 0);
    ctl->arrive = 0;
    __threadfence();
  }
}

// ---------------------------------------------------------------------------- coefficient freeze
// The first frozen-coefficient mean round after the joint rounds, fused with the
// freeze: from round T's precision state ({P~, h~} ring and P chain) it writes
//   c_out = c_ik = -A / (P~_i - P_ki),  c_in = c_ki = -A / (P~_k - c_out A),  1/P~_i
// and uses them at once for mean round T + 1, the sender's {P~_k, h~_k} coming
// from ONE 8-byte gather (the separate freeze pass would re-read every slot and
// gather P~_k).  Same arithmetic as k32_coef followed by k32_mean.  If the mean
// solve is already decided (T reached the inner cap) only the coefficients and
// 1/P~ are written.
template <int L, int U>
__global__ void __launch_bounds__(kBlock) k32_freeze(Args32 a) {
  DevCtl *ctl = a.ctl;
  const bool coef_only = ctl->done;
  const int T = ctl->round, t = T + 1;
  const float *__restrict__ Ms = (T & 1) ? a.MP1 : a.MP0;  // P_ki of round T
  const float2 *__restrict__ QT = ring3(a.NQ0, a.NQ1, a.NQ2, T);
  float *__restrict__ Hc = (t & 1) ? a.H1 : a.H0;  // holds t-2, becomes t
  const float *__restrict__ Hm2 = ring3(a.NH0, a.NH1, a.NH2, t + 1);
  float *__restrict__ Ht = ring3(a.NH0, a.NH1, a.NH2, t);
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  float dxx = 0.f, xx = 0.f;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int i = base + sw;
    float acc = 0.f;
    float2 qi = make_float2(1.f, 0.f);
    float rhs_i = 0.f;
    if (i < a.n) {
      qi = QT[i];
      const float hi2 = t >= 2 ? Hm2[i] : 0.f;
      rhs_i = a.rhs[i];  // requested before the slots (latency overlap)
      const int e1 = a.rp[i + 1];
      for (int eb = a.rp[i] + sl; eb < e1; eb += L * U) {
        int k[U];
        float A[U], Ps[U], hs[U];
        float2 qk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = eb + u * L;
          if (e < e1) { k[u] = __ldcs(a.ci + e); A[u] = __ldcs(a.av + e); Ps[u] = __ldcs(Ms + e); hs[u] = __ldcs(Hc + e); }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (eb + u * L < e1) qk[u] = __ldcg(QT + k[u]);  // random gather, L2 only
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = eb + u * L;
          if (e < e1) {
            const float cout = -A[u] / (qi.x - Ps[u]);
            const float Pout = cout * A[u];
            const float cin = -A[u] / (qk[u].x - Pout);
            a.CF[e] = make_float2(cin, cout);
            if (!coef_only) {
              const float hout = t >= 2 ? cout * (hi2 - hs[u]) : 0.f;  // message i -> k at t-1
              const float hn = cin * (qk[u].y - hout);                 // message k -> i at t
              __stcs(Hc + e, hn);
              acc += hn;
            }
          }
        }
      }
    }
    acc = sub_sum<L>(acc);
    if (i < a.n && sl == 0) {
      const float ip = 1.f / qi.x;
      a.invP[i] = ip;
      if (!coef_only) {
        const float hnew = rhs_i + acc;
        Ht[i] = hnew;
        const float x = hnew * ip, dx = (hnew - qi.y) * ip;
        dxx = fmaf(dx, dx, dxx);
        xx = fmaf(x, x, xx);
      }
    }
  }
  if (coef_only) return;
  double v[2] = {(double)dxx, (double)xx}, tot[2];
  const int modes[2] = {0, 0};
  block_sum<2>(v);
  if (last_block_reduce<2>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    ctl->round = t;
    ctl->rr = tot[0];
    ctl->xx = tot[1];
    if (!isfinite(tot[0]) || !isfinite(tot[1])) {
      ctl->status = GABP_DIVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (t >= 2 && tot[0] <= ctl->tol2bb * tot[1]) {
      ctl->status = GABP_OK; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (t >= ctl->max_iter) {
      ctl->status = GABP_NOT_CONVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    }
    if (a.use_cond && ctl->done) cudaGraphSetConditional(a.cond, 0);
    ctl->arrive = 0;
    __threadfence();
  }
}

// ---------------------------------------------------------------------------- FP64 outer steps
// r = b - A x over the full CSR (diagonal included), in FP64; the FP32 copy of r
// seeds the next inner solve (its round-0 aggregate h~^(0) = r and its RHS).
template <int L>
__global__ void __launch_bounds__(kBlock) k64_residual(int n, const int *__restrict__ rowptr,
                                                       const int *__restrict__ col, const double *__restrict__ val,
                                                       const double *__restrict__ b, const double *__restrict__ x,
                                                       float *__restrict__ rhs32, float *__restrict__ nh0,
                                                       DevCtl *ctl, double *partials, int set_bb,
                                                       const int *skip = nullptr, int x_zero = 0) {
  if (skip && *skip) return;  // device-loop graph: the loop already stopped
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  constexpr int U = 4;  // entries per lane whose loads are issued together
  double rr = 0.0;
  for (int base = warp * RPW; base < n; base += nwarps * RPW) {
    const int i = base + sw;
    double ax = 0.0, bi = 0.0;
    if (i < n) {
      bi = b[i];  // requested before the row's entries (latency overlap)
      if (!x_zero) {  // x = 0 (the first residual): r = b exactly, no product needed
        const int p1 = rowptr[i + 1];
        for (int pb = rowptr[i] + sl; pb < p1; pb += L * U) {
          int c[U];
          double v[U], xc[U];
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (pb + u * L < p1) { c[u] = __ldcs(col + pb + u * L); v[u] = __ldcs(val + pb + u * L); }
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (pb + u * L < p1) xc[u] = __ldcg(x + c[u]);  // random gather, L2 only
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (pb + u * L < p1) ax = fma(v[u], xc[u], ax);
        }
      }
    }
    ax = sub_sum<L>(ax);
    if (i < n && sl == 0) {
      const double r = bi - ax;
      rr = fma(r, r, rr);
      const float rf = (float)r;
      rhs32[i] = rf;
      nh0[i] = rf;
    }
  }
  double v[1] = {rr}, tot[1];
  const int modes[1] = {0};
  block_sum<1>(v);
  if (last_block_reduce<1>(v, modes, partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    ctl->rr = tot[0];
    if (set_bb) {
      ctl->bb = tot[0];
    }
    ctl->arrive = 0;
    __threadfence();
  }
}

// x <- x + d, d_i = h~_i / P~_i of the inner solve's final round (FP64 accumulate).
__global__ void k64_update(int n, double *__restrict__ x, const float *__restrict__ hT,
                           const float *__restrict__ invP) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += (double)(hT[i] * invP[i]);
}

__global__ void k_to_f32(int64_t m, const double *__restrict__ s, float *__restrict__ d) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) d[i] = (float)s[i];
}

__global__ void k_diag32(int n, const double *__restrict__ ad, const double *__restrict__ gam,
                         float *__restrict__ d32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d32[i] = (float)(ad[i] + (gam ? gam[i] : 0.0));
}

__global__ void k_ctl_reset(DevCtl *c, int max_iter, double tol2, int round0 = 0) {
  c->round = round0;
  c->done = round0 > 0 && round0 >= max_iter;
  c->status = GABP_NOT_CONVERGED;
  c->iters = round0;
  c->result_round = round0;
  c->max_iter = max_iter;
  c->check_from = 1;
  c->stable = 0;
  c->tol2bb = tol2;
  c->rr = 0.0;
  c->xx = 0.0;
  c->maxrel = 0.0;
  c->arrive = 0;
  c->edge_bad = 0;
  c->no_stop = 0;
}

// Diagonal loading of the convergence fix.  mode 1: Gamma_i = gamma A_ii (the
// unit-diagonal model I - R loaded by gamma I, in A's scaling; walk-summable for
// gamma > rho(|R|) - 1).  mode 2: Gamma_i = max(0, sum_j |A_ij| - A_ii) + gamma A_ii,
// which makes A + Gamma diagonally dominant for gamma > 0.
__global__ void k_gamma(int n, int mode, double gamma, const int *__restrict__ rp, const double *__restrict__ av,
                        const double *__restrict__ ad, double *__restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = ad[i];
  if (mode == 1) {
    out[i] = gamma * d;
  } else {
    double s = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) s += fabs(av[e]);
    out[i] = fmax(0.0, s - d) + gamma * d;
  }
}

__global__ void k32_marginals(int n, const float *__restrict__ P, double *__restrict__ Pi) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Pi[i] = (double)P[i];
}

// ---------------------------------------------------------------------------- host side
gabp_status make_gamma(gabp_handle h, double *out) {
  Graph &g = h->g;
  k_gamma<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, h->opt.gamma_mode, h->opt.gamma, g.rp, g.av,
                                                                   g.ad, out);
  GABP_CUDA(cudaGetLastError());
  return GABP_OK;
}

gabp_status marginals32(gabp_handle h, double *Pi) {
  Work32 &w = h->w32;
  if (!w.MP[0] || w.prec_round < 0) return GABP_ERR_INVALID;
  Graph &g = h->g;
  const float *P = w.NP[w.prec_round % 3];
  k32_marginals<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, P, Pi);
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return GABP_OK;
}

gabp_status ensure_w32(gabp_handle h, int R) {
  Work32 &w = h->w32;
  Graph &g = h->g;
  size_t E = (size_t)(g.E > 0 ? g.E : 1), n = (size_t)g.n;
  if (!w.MP[0]) {
    GABP_CUDA(cudaMalloc(&w.MP[0], sizeof(float) * E));
    GABP_CUDA(cudaMalloc(&w.MP[1], sizeof(float) * E));
    for (int j = 0; j < 3; ++j) GABP_CUDA(cudaMalloc(&w.NP[j], sizeof(float) * n));
    GABP_CUDA(cudaMalloc(&w.CF, sizeof(float2) * E));
    GABP_CUDA(cudaMalloc(&w.invP, sizeof(float) * n));
    GABP_CUDA(cudaMalloc(&g.av32, sizeof(float) * E));
    GABP_CUDA(cudaMalloc(&g.ad32, sizeof(float) * n));
    GABP_CUDA(cudaMalloc(&w.ctlR, sizeof(DevCtl)));
    GABP_CUDA(cudaMemsetAsync(w.ctlR, 0, sizeof(DevCtl), h->stream));
    for (int j = 0; j < 3; ++j) GABP_CUDA(cudaMalloc(&w.NQ[j], sizeof(float2) * n));
    k_to_f32<<<(int)((E + kBlock - 1) / kBlock), kBlock, 0, h->stream>>>((int64_t)g.E, g.av, g.av32);
    GABP_CUDA(cudaGetLastError());
  }
  if (w.R < R) {
    cudaFree(w.H[0]); cudaFree(w.H[1]);
    for (int j = 0; j < 3; ++j) cudaFree(w.NH[j]);
    cudaFree(w.rhs32); cudaFree(w.X); cudaFree(w.Rs); cudaFree(w.Bt);
    w.H[0] = w.H[1] = nullptr;
    w.NH[0] = w.NH[1] = w.NH[2] = nullptr;
    w.rhs32 = nullptr; w.X = w.Rs = w.Bt = nullptr;
    w.R = 0;
    GABP_CUDA(cudaMalloc(&w.H[0], sizeof(float) * E * R));
    GABP_CUDA(cudaMalloc(&w.H[1], sizeof(float) * E * R));
    for (int j = 0; j < 3; ++j) GABP_CUDA(cudaMalloc(&w.NH[j], sizeof(float) * n * R));
    GABP_CUDA(cudaMalloc(&w.rhs32, sizeof(float) * n * R));
    GABP_CUDA(cudaMalloc(&w.X, sizeof(double) * n * R));
    w.R = R;
    if (h->gH32) cudaGraphExecDestroy(h->gH32);
    h->gH32 = nullptr;
    h->gH32_R = -1;
    if (h->gRef) cudaGraphExecDestroy(h->gRef);  // holds the old buffers
    if (h->gRefG) cudaGraphDestroy(h->gRefG);
    h->gRef = nullptr;
    h->gRefG = nullptr;
    h->gRef_key = -1;
  }
  return GABP_OK;
}

void free_w32(gabp_handle h) {
  Work32 &w = h->w32;
  cudaFree(w.MP[0]); cudaFree(w.MP[1]);
  for (int j = 0; j < 3; ++j) { cudaFree(w.NP[j]); cudaFree(w.NH[j]); cudaFree(w.NQ[j]); }
  cudaFree(w.CF); cudaFree(w.invP); cudaFree(w.H[0]); cudaFree(w.H[1]);
  cudaFree(w.rhs32); cudaFree(w.X); cudaFree(w.Rs); cudaFree(w.Bt); cudaFree(w.colnorm);
  cudaFree(w.ctlR); cudaFree(w.rhs_active); cudaFree(w.rc); cudaFree(w.Bd);
  if (w.rc_host) cudaFreeHost(w.rc_host);
  w = Work32{};
}

static Args32 args32(gabp_handle h) {
  Args32 a;
  Graph &g = h->g;
  Work32 &w = h->w32;
  a.n = g.n; a.rp = g.rp; a.ci = g.ci; a.av = g.av32; a.ad = g.ad32;
  a.dense = g.n > 1 && (int64_t)g.E == (int64_t)g.n * (g.n - 1);  // every off-diagonal entry stored
  a.MP0 = w.MP[0]; a.MP1 = w.MP[1];
  a.NP0 = w.NP[0]; a.NP1 = w.NP[1]; a.NP2 = w.NP[2];
  a.CF = w.CF; a.invP = w.invP;
  a.H0 = w.H[0]; a.H1 = w.H[1];
  a.NH0 = w.NH[0]; a.NH1 = w.NH[1]; a.NH2 = w.NH[2];
  a.rhs = w.rhs32;
  a.NQ0 = w.NQ[0]; a.NQ1 = w.NQ[1]; a.NQ2 = w.NQ[2];
  a.cond = 0;
  a.use_cond = 0;
  a.ctl = h->ctl;
  a.partials = h->partials;
  return a;
}

// A mean round of shape (LL, UU) on stream st: the complete-pattern variant when the
// matrix is dense.
template <int LL, int UU>
static void launch_mean(gabp_handle h, const Args32 &a, cudaStream_t st) {
  const int n = h->g.n;
  if (a.dense)
    k32_mean<LL, UU, true><<<blocks_for(n, kBlock / LL, resident_grid(h->num_sms, k32_mean<LL, UU, true>)), kBlock, 0,
                             st>>>(a);
  else
    k32_mean<LL, UU><<<blocks_for(n, kBlock / LL, resident_grid(h->num_sms, k32_mean<LL, UU>)), kBlock, 0, st>>>(a);
}

// Shape (lanes per row, unroll) of an FP32 round kernel: the option if set, else
// the autotuned one, else a heuristic (one unrolled pass of 4 slots per lane
// covers a row of average degree).
enum { K32_PREC = 0, K32_MEAN = 1, K32_JOINT = 2 };
static int &tuned32(gabp_handle h, int kind) {
  return kind == K32_MEAN ? h->tuned_Lm32 : kind == K32_JOINT ? h->tuned_Lj32 : h->tuned_Lp32;
}
static int shape32(gabp_handle h, int kind) {
  if (h->opt.lanes) return pinned_shape32(h->opt.lanes, h->opt.unroll);  // validated by the option check
  const int tuned = tuned32(h, kind);
  if (tuned) return tuned;
  double d = h->g.avg_deg;
  int L = 1;
  while (L < 8 && (2 * L) * kUnroll32 <= d + 0.5) L *= 2;
  return shape_code(L, kUnroll32);
}

// Autotuner of the FP32 round kernels' shapes: a few rounds of every candidate
// (lanes, unroll) under a scratch control block, fastest kept.
static gabp_status autotune32(gabp_handle h, int kind) {
  if (h->opt.lanes || tuned32(h, kind)) return GABP_OK;
  Graph &g = h->g;
  gabp_status s0 = tune_ctl(h, nullptr);  // allocates the scratch control block on first use
  if (s0 != GABP_OK) return s0;
  Args32 a = args32(h);
  a.ctl = h->ctl_tune;
  float best = 1e30f;
  int bestS = kShapes[0];
  gabp_status s;
  for (int sc : kShapes) {
    if ((s = tune_ctl(h, nullptr)) != GABP_OK) return s;
    float ms = 1e30f;
    with_shape(sc, [&](auto Lc, auto Uc) {
      constexpr int LL = decltype(Lc)::value, UU = decltype(Uc)::value;
      if (kind == K32_MEAN)
        ms = time_launches(h, [&] { launch_mean<LL, UU>(h, a, h->stream); }, 5);
      else if (kind == K32_JOINT)
        ms = time_launches(h, [&] {
          k32_joint<LL, UU><<<blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, k32_joint<LL, UU>)), kBlock, 0,
                              h->stream>>>(a);
        }, 5);
      else
        ms = time_launches(h, [&] {
          k32_prec<LL, UU><<<blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, k32_prec<LL, UU>)), kBlock, 0,
                             h->stream>>>(a);
        }, 5);
    });
    if (ms < best) { best = ms; bestS = sc; }
  }
  GABP_CUDA(cudaGetLastError());
  tuned32(h, kind) = bestS;
  tune_cache_store(h);
  return GABP_OK;
}

gabp_status precision_phase32(gabp_handle h, const double *gamma_diag) {
  NvtxRange nvtx_("gabp fp32 precision rounds");
  Work32 &w = h->w32;
  Graph &g = h->g;
  size_t E = (size_t)(g.E > 0 ? g.E : 1);
  k_diag32<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, g.ad, gamma_diag, g.ad32);
  // round-0 state: zero precision messages, P~ = diagonal
  auto init = [&]() -> gabp_status {
    GABP_CUDA(cudaMemsetAsync(w.MP[0], 0, sizeof(float) * E, h->stream));
    GABP_CUDA(cudaMemsetAsync(w.MP[1], 0, sizeof(float) * E, h->stream));
    GABP_CUDA(cudaMemcpyAsync(w.NP[0], g.ad32, sizeof(float) * g.n, cudaMemcpyDeviceToDevice, h->stream));
    return GABP_OK;
  };
  gabp_status st = init();
  if (st != GABP_OK) return st;
  if (!h->opt.lanes && !h->tuned_Lp32) {
    if ((st = autotune32(h, K32_PREC)) != GABP_OK) return st;
    if ((st = init()) != GABP_OK) return st;
  }
  const int SH = shape32(h, K32_PREC);
  k_ctl_reset<<<1, 1, 0, h->stream>>>(h->ctl, kPrecMaxRounds, std::ldexp(1.0, -h->opt.prec_stop_log2));
  h->prof.launches += 2;
  GABP_CUDA(cudaGetLastError());
  Args32 a = args32(h);
  gabp_status s;
  with_shape(SH, [&](auto Lc, auto Uc) {
    constexpr int LL = decltype(Lc)::value, UU = decltype(Uc)::value;
    s = run_rounds(h, &h->gP32, &h->gP32_L, SH, [&] {
      const int nb = blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, k32_prec<LL, UU>));
      k32_prec<LL, UU><<<nb, kBlock, 0, h->stream>>>(a);
    }, kPrecMaxRounds, PH_PREC32);
  });
  if (s != GABP_OK) return s;
  const DevCtl c = *h->ctl_host;
  h->stats.rounds += c.round;
  if (c.status == GABP_BREAKDOWN || c.status == GABP_DIVERGED) return (gabp_status)c.status;
  const int Lc = SH & 0xff;
  GABP_DISPATCH_L(Lc, (k32_coef<LL><<<blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, k32_coef<LL>)), kBlock, 0,
                                      h->stream>>>(a, c.result_round)));
  h->prof.launches += 1;
  GABP_CUDA(cudaGetLastError());
  w.prec_round = c.result_round;
  w.coef_ready = true;
  return GABP_OK;
}

// Joint rounds (precision and mean messages together) from zero messages until
// the precisions are stationary or `cap` rounds; returns that round T, whose
// state freeze32 freezes.  The mean state of round T is the start of the first
// inner solve's frozen-coefficient rounds.  Needs rhs32 / NH[0] = r (k64_residual).
static gabp_status joint_phase32(gabp_handle h, const double *gamma_diag, int cap, int *T_out) {
  Work32 &w = h->w32;
  Graph &g = h->g;
  size_t E = (size_t)(g.E > 0 ? g.E : 1);
  k_diag32<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, g.ad, gamma_diag, g.ad32);
  auto init = [&]() -> gabp_status {
    GABP_CUDA(cudaMemsetAsync(w.MP[0], 0, sizeof(float) * E, h->stream));
    GABP_CUDA(cudaMemsetAsync(w.MP[1], 0, sizeof(float) * E, h->stream));
    GABP_CUDA(cudaMemsetAsync(w.H[0], 0, sizeof(float) * E, h->stream));
    k32_joint_init<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, g.ad32, w.rhs32, w.NQ[0], w.NP[0]);
    GABP_CUDA(cudaGetLastError());
    return GABP_OK;
  };
  gabp_status st = init();
  if (st != GABP_OK) return st;
  if (!h->opt.lanes && !h->tuned_Lj32) {
    if ((st = autotune32(h, K32_JOINT)) != GABP_OK) return st;
    if ((st = init()) != GABP_OK) return st;
  }
  const int SH = shape32(h, K32_JOINT);
  const int rounds = std::max(1, std::min(kPrecMaxRounds, cap));
  k_ctl_reset<<<1, 1, 0, h->stream>>>(h->ctl, rounds, std::ldexp(1.0, -h->opt.prec_stop_log2));
  h->prof.launches += 3;
  GABP_CUDA(cudaGetLastError());
  Args32 a = args32(h);
  gabp_status s;
  with_shape(SH, [&](auto Lc, auto Uc) {
    constexpr int LL = decltype(Lc)::value, UU = decltype(Uc)::value;
    s = run_rounds(h, &h->gJ32, &h->gJ32_L, SH, [&] {
      const int nb = blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, k32_joint<LL, UU>));
      k32_joint<LL, UU><<<nb, kBlock, 0, h->stream>>>(a);
    }, rounds, PH_PREC32);
  });
  if (s != GABP_OK) return s;
  const DevCtl c = *h->ctl_host;
  if (c.status == GABP_BREAKDOWN || c.status == GABP_DIVERGED) return (gabp_status)c.status;
  *T_out = c.result_round;
  return GABP_OK;
}

// The coefficient freeze at the joint rounds' last round T fused with mean round
// T + 1 (k32_freeze), on the control block armed for the inner solve from T.
static gabp_status freeze32(gabp_handle h, int T) {
  Graph &g = h->g;
  Work32 &w = h->w32;
  Args32 a = args32(h);
  const int SH = shape32(h, K32_JOINT);
  prof_begin(h);
  with_shape(SH, [&](auto Lc, auto Uc) {
    constexpr int LL = decltype(Lc)::value, UU = decltype(Uc)::value;
    k32_freeze<LL, UU><<<blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, k32_freeze<LL, UU>)), kBlock, 0,
                         h->stream>>>(a);
  });
  prof_end(h);
  GABP_CUDA(cudaGetLastError());
  prof_collect(h, PH_FREEZE32, 1);
  h->prof.launches += 1;
  w.prec_round = T;
  w.coef_ready = true;
  return GABP_OK;
}

// ---------------------------------------------------------------------------- device-driven refinement loop
// The whole FP32 + FP64-refinement solve of one right-hand side as ONE CUDA
// graph: the stop decisions that the host loop of solve32_refine takes after
// each batch of rounds and after each residual are taken by single-thread
// kernels that set the conditions of while / if nodes (cudaGraphSetConditional),
// so the host only launches the graph and reads the result:
//
//   r = b - A x (x = 0), decide
//   while (refining) {
//     zero the inner messages
//     if (precisions not computed yet) { joint rounds while not stationary; freeze; continue at T }
//     while (inner not decided) { K frozen-coefficient mean rounds }
//     x += d; r = b - A x; decide
//   }
//
// Same arithmetic, same kernels, same decisions as the host-driven loop.
struct RefineCtl {
  // parameters of the call
  double tol, tol2, inner_tol, prec_thr;
  int max_refine, max_iter, inner_max, prec_cap;
  // loop state
  double rr, bb, it2;
  int steps, total_inner, status, skip, joint_pending, prec_round, cap;
  int joint_rounds; // rounds the joint loop ran
  int launches;     // kernels the graph launched after its first residual and decision
  int inner_start;  // round at which the current inner solve's while loop starts
};

struct RefineParams {
  double tol, inner_tol, prec_thr;
  int max_refine, max_iter, inner_max, prec_cap, joint;
};

__device__ void ctl_arm(DevCtl *c, int round0, int max_iter, double tol2) {
  c->round = round0;
  c->done = round0 >= max_iter;
  c->status = GABP_NOT_CONVERGED;
  c->iters = round0;
  c->result_round = round0;
  c->max_iter = max_iter;
  c->check_from = 1;
  c->stable = 0;
  c->tol2bb = tol2;
  c->rr = 0.0;
  c->xx = 0.0;
  c->maxrel = 0.0;
  c->arrive = 0;
  c->edge_bad = 0;
  c->no_stop = 0;
}

__global__ void k_ref_setup(RefineCtl *rc, RefineParams p) {
  RefineCtl r = {};
  r.tol = p.tol;
  r.tol2 = p.tol * p.tol;
  r.inner_tol = p.inner_tol;
  r.prec_thr = p.prec_thr;
  r.max_refine = p.max_refine;
  r.max_iter = p.max_iter;
  r.inner_max = p.inner_max;
  r.prec_cap = p.prec_cap;
  r.status = GABP_NOT_CONVERGED;
  r.joint_pending = p.joint;
  r.prec_round = -1;
  *rc = r;
}

// After a residual: stop (converged / diverged / caps) or arm the next inner solve.
__global__ void k_ref_decide(RefineCtl *rc, const DevCtl *ctlR, DevCtl *ctl, int first,
                             cudaGraphConditionalHandle h_outer, cudaGraphConditionalHandle h_joint,
                             cudaGraphConditionalHandle h_inner) {
  int go = 0;
  if (!rc->skip) {
    if (!first) rc->steps += 1;
    const double rr = ctlR->rr, bb = ctlR->bb;
    rc->rr = rr;
    rc->bb = bb;
    if (!isfinite(rr)) rc->status = GABP_DIVERGED;
    else if (bb == 0.0 || rr <= rc->tol2 * bb) rc->status = GABP_OK;
    else if (rc->steps >= rc->max_refine || rc->total_inner >= rc->max_iter) rc->status = GABP_NOT_CONVERGED;
    else {
      go = 1;
      rc->inner_start = 0;
      rc->cap = min(rc->inner_max, max(1, rc->max_iter - rc->total_inner));
      const double it = inner_target(rc->inner_tol, rc->tol, bb, rr);
      rc->it2 = it * it;
      ctl_arm(ctl, 0, rc->cap, rc->it2);
    }
  }
  cudaGraphSetConditional(h_outer, go);
  cudaGraphSetConditional(h_joint, go && rc->joint_pending);
  cudaGraphSetConditional(h_inner, go);
}

__global__ void k_joint_prep(RefineCtl *rc, DevCtl *ctl, cudaGraphConditionalHandle h_jw) {
  ctl_arm(ctl, 0, max(1, min(rc->prec_cap, rc->cap)), rc->prec_thr);
  cudaGraphSetConditional(h_jw, 1);
}

// After the joint rounds (and the freeze at their last round T): stop on a
// breakdown, else continue the first inner solve's rounds from T.
__global__ void k_joint_after(RefineCtl *rc, DevCtl *ctl, cudaGraphConditionalHandle h_inner) {
  const int T = ctl->result_round, st = ctl->status;
  rc->joint_pending = 0;
  rc->joint_rounds = ctl->round;
  if (st == GABP_BREAKDOWN || st == GABP_DIVERGED) {
    rc->status = st;
    rc->skip = 1;
    cudaGraphSetConditional(h_inner, 0);
    return;
  }
  rc->prec_round = T;
  ctl_arm(ctl, T, rc->cap, rc->it2);
  cudaGraphSetConditional(h_inner, T < rc->cap);
}

// kLoopK round kernels per while-body iteration (later ones exit at once when decided)
constexpr int kLoopK = 2;

// The joint rounds' while loop ran ceil(rounds / kLoopK) bodies; with the prep, the
// joint-after, the freeze and this kernel: the launches of the joint block.  Marks
// the round from which the first inner solve's loop continues.
__global__ void k_joint_mark(RefineCtl *rc, const DevCtl *ctl) {
  rc->launches += 2 + 2 + 1 + kLoopK * ((rc->joint_rounds + kLoopK - 1) / kLoopK);
  rc->inner_start = ctl->round;
}

__global__ void k_ref_after_inner(RefineCtl *rc, const DevCtl *ctl) {
  // this step's inner loop ran ceil(rounds / kLoopK) bodies; then this kernel, the
  // update, the residual and the decision
  const int worked = max(0, ctl->round - rc->inner_start);
  rc->launches += kLoopK * ((worked + kLoopK - 1) / kLoopK) + 4;
  rc->inner_start = ctl->round;
  if (rc->skip) return;
  rc->total_inner += ctl->result_round;
  if (ctl->status == GABP_DIVERGED) {
    rc->status = GABP_DIVERGED;
    rc->skip = 1;
  }
}

// x <- x + d with d from the inner solve's final round (read on the device)
__global__ void k64_update_ctl(int n, double *__restrict__ x, const float *NH0, const float *NH1, const float *NH2,
                               const float *__restrict__ invP, const DevCtl *ctl, const int *skip) {
  if (*skip) return;
  const int m = ctl->result_round % 3;
  const float *__restrict__ hT = m == 0 ? NH0 : (m == 1 ? NH1 : NH2);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += (double)(hT[i] * invP[i]);
}

// A graph under construction: nodes are appended in sequence after `last`.
struct SeqGraph {
  cudaGraph_t g;
  cudaGraphNode_t last;
};

// Append the launches `f` makes on `stream`, captured, after seq.last.
template <typename F>
static cudaError_t seq_capture(SeqGraph &seq, cudaStream_t stream, F &&f) {
  cudaError_t e = cudaStreamBeginCaptureToGraph(stream, seq.g, seq.last ? &seq.last : nullptr, nullptr,
                                                seq.last ? 1 : 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  f();
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  e = cudaStreamGetCaptureInfo(stream, &cs, nullptr, nullptr, &deps, nullptr, &nd);
  std::vector<cudaGraphNode_t> frontier(deps, deps + (e == cudaSuccess ? nd : 0));
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(stream, &out);
  if (e != cudaSuccess) return e;
  if (e2 != cudaSuccess) return e2;
  if (frontier.size() == 1) {
    seq.last = frontier[0];
  } else if (frontier.size() > 1) {
    cudaGraphNode_t join;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeEmpty;
    e = cudaGraphAddNode(&join, seq.g, frontier.data(), nullptr, frontier.size(), &p);
    if (e != cudaSuccess) return e;
    seq.last = join;
  }
  return cudaSuccess;
}

// Append a while / if node on `handle`; returns its body as a new sequence.
static cudaError_t seq_conditional(SeqGraph &seq, cudaGraphConditionalHandle handle, cudaGraphConditionalNodeType type,
                                   SeqGraph *body) {
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = handle;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphAddNode(&node, seq.g, seq.last ? &seq.last : nullptr, nullptr, seq.last ? 1 : 0, &p);
  if (e != cudaSuccess) return e;
  seq.last = node;
  body->g = p.conditional.phGraph_out[0];
  body->last = nullptr;
  return cudaSuccess;
}

static gabp_status build_refine_graph(gabp_handle h, int SHm, int SHj, int LR) {
  Graph &g = h->g;
  Work32 &w = h->w32;
  const size_t E = (size_t)(g.E > 0 ? g.E : 1);
  cudaStream_t st = h->stream;
  cudaGraph_t root;
  GABP_CUDA(cudaGraphCreate(&root, 0));
  struct Guard {
    cudaGraph_t *g;
    ~Guard() { if (*g) cudaGraphDestroy(*g); }
  } guard{&root};
  cudaGraphConditionalHandle h_outer, h_joint, h_jw, h_inner;
  GABP_CUDA(cudaGraphConditionalHandleCreate(&h_outer, root, 0, cudaGraphCondAssignDefault));
  GABP_CUDA(cudaGraphConditionalHandleCreate(&h_joint, root, 0, cudaGraphCondAssignDefault));
  GABP_CUDA(cudaGraphConditionalHandleCreate(&h_jw, root, 0, cudaGraphCondAssignDefault));
  GABP_CUDA(cudaGraphConditionalHandleCreate(&h_inner, root, 0, cudaGraphCondAssignDefault));
  Args32 a = args32(h);
  int nbr = 1;
  GABP_DISPATCH_L(LR, nbr = blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, k64_residual<LL>)));
  RefineCtl *rc = w.rc;
  const int nb1 = (g.n + kBlock - 1) / kBlock;
  auto residual = [&](int first) {
    GABP_DISPATCH_L(LR, (k64_residual<LL><<<nbr, kBlock, 0, st>>>(g.n, g.rowptr, g.col, g.val, w.Bd, w.X, w.rhs32,
                                                                    w.NH[0], w.ctlR, h->partials, first,
                                                                    &rc->skip, first)));
  };
  SeqGraph top{root, nullptr};
  cudaError_t e = seq_capture(top, st, [&] {
    cudaMemsetAsync(w.X, 0, sizeof(double) * g.n, st);
    residual(1);
    k_ref_decide<<<1, 1, 0, st>>>(rc, w.ctlR, h->ctl, 1, h_outer, h_joint, h_inner);
  });
  SeqGraph outer{}, joint{}, jw{}, inner{};
  if (e == cudaSuccess) e = seq_conditional(top, h_outer, cudaGraphCondTypeWhile, &outer);
  if (e == cudaSuccess)
    e = seq_capture(outer, st, [&] { cudaMemsetAsync(w.H[0], 0, sizeof(float) * E, st); });
  // precision state computed together with the first inner solve
  if (e == cudaSuccess) e = seq_conditional(outer, h_joint, cudaGraphCondTypeIf, &joint);
  if (e == cudaSuccess)
    e = seq_capture(joint, st, [&] {
      cudaMemsetAsync(w.MP[0], 0, sizeof(float) * E, st);
      cudaMemsetAsync(w.MP[1], 0, sizeof(float) * E, st);
      k32_joint_init<<<nb1, kBlock, 0, st>>>(g.n, g.ad32, w.rhs32, w.NQ[0], w.NP[0]);
      k_joint_prep<<<1, 1, 0, st>>>(rc, h->ctl, h_jw);
    });
  if (e == cudaSuccess) e = seq_conditional(joint, h_jw, cudaGraphCondTypeWhile, &jw);
  if (e == cudaSuccess)
    e = seq_capture(jw, st, [&] {
      Args32 aj = a;
      aj.cond = h_jw;
      aj.use_cond = 1;
      with_shape(SHj, [&](auto Lc, auto Uc) {
        constexpr int LL = decltype(Lc)::value, UU = decltype(Uc)::value;
        const int nb = blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, k32_joint<LL, UU>));
        for (int k = 0; k < kLoopK; ++k) k32_joint<LL, UU><<<nb, kBlock, 0, st>>>(aj);
      });
    });
  if (e == cudaSuccess)
    e = seq_capture(joint, st, [&] {
      k_joint_after<<<1, 1, 0, st>>>(rc, h->ctl, h_inner);
      // freeze at T fused with round T + 1 (only the freeze if the inner cap is reached)
      Args32 af = a;
      af.cond = h_inner;
      af.use_cond = 1;
      with_shape(SHj, [&](auto Lc, auto Uc) {
        constexpr int LL = decltype(Lc)::value, UU = decltype(Uc)::value;
        k32_freeze<LL, UU><<<blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, k32_freeze<LL, UU>)), kBlock, 0,
                             st>>>(af);
      });
      k_joint_mark<<<1, 1, 0, st>>>(rc, h->ctl);
    });
  // the inner solve's frozen-coefficient rounds
  if (e == cudaSuccess) e = seq_conditional(outer, h_inner, cudaGraphCondTypeWhile, &inner);
  if (e == cudaSuccess)
    e = seq_capture(inner, st, [&] {
      Args32 am = a;
      am.cond = h_inner;
      am.use_cond = 1;
      with_shape(SHm, [&](auto Lc, auto Uc) {
        constexpr int LL = decltype(Lc)::value, UU = decltype(Uc)::value;
        for (int k = 0; k < kLoopK; ++k) launch_mean<LL, UU>(h, am, st);
      });
    });
  if (e == cudaSuccess)
    e = seq_capture(outer, st, [&] {
      k_ref_after_inner<<<1, 1, 0, st>>>(rc, h->ctl);
      k64_update_ctl<<<nb1, kBlock, 0, st>>>(g.n, w.X, w.NH[0], w.NH[1], w.NH[2], w.invP, h->ctl, &rc->skip);
      residual(0);
      k_ref_decide<<<1, 1, 0, st>>>(rc, w.ctlR, h->ctl, 0, h_outer, h_joint, h_inner);
    });
  if (e != cudaSuccess) return cuda_fail(e, "build the refinement-loop graph");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, root, 0);
  if (e != cudaSuccess) return cuda_fail(e, "instantiate the refinement-loop graph");
  if (h->gRef) cudaGraphExecDestroy(h->gRef);
  if (h->gRefG) cudaGraphDestroy(h->gRefG);
  h->gRef = exec;
  h->gRefG = root;
  root = nullptr;
  return GABP_OK;
}

// solve32_refine for one right-hand side without loading, as one graph launch.
static gabp_status solve32_device_loop(gabp_handle h, const double *B, double *X, double tol, int max_iter,
                                       int *iters, double *relres) {
  Work32 &w = h->w32;
  Graph &g = h->g;
  if (!w.rc) {
    GABP_CUDA(cudaMalloc(&w.rc, sizeof(RefineCtl)));
    GABP_CUDA(cudaMallocHost(&w.rc_host, sizeof(RefineCtl)));
    GABP_CUDA(cudaMalloc(&w.Bd, sizeof(double) * (size_t)g.n));
  }
  const bool joint = !w.coef_ready || !h->opt.reuse_precisions;
  if (joint) {
    w.coef_ready = false;
    if (!h->opt.overlap_precision) {
      gabp_status s = precision_phase32(h, nullptr);
      if (s != GABP_OK) return s;
    } else {
      k_diag32<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, g.ad, nullptr, g.ad32);
      GABP_CUDA(cudaGetLastError());
      if (!h->opt.lanes && !h->tuned_Lj32) {
        // the autotuner runs a few joint rounds on scratch state (re-initialised by the graph)
        const size_t E = (size_t)(g.E > 0 ? g.E : 1);
        GABP_CUDA(cudaMemsetAsync(w.rhs32, 0, sizeof(float) * g.n, h->stream));
        GABP_CUDA(cudaMemsetAsync(w.MP[0], 0, sizeof(float) * E, h->stream));
        GABP_CUDA(cudaMemsetAsync(w.MP[1], 0, sizeof(float) * E, h->stream));
        GABP_CUDA(cudaMemsetAsync(w.H[0], 0, sizeof(float) * E, h->stream));
        k32_joint_init<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, g.ad32, w.rhs32, w.NQ[0], w.NP[0]);
        gabp_status s = autotune32(h, K32_JOINT);
        if (s != GABP_OK) return s;
      }
    }
  }
  const bool run_joint = joint && h->opt.overlap_precision;
  gabp_status s = autotune32(h, K32_MEAN);
  if (s != GABP_OK) return s;
  const int SHm = shape32(h, K32_MEAN), SHj = shape32(h, K32_JOINT);
  const int LR = h->opt.lanes ? h->opt.lanes : (g.avg_deg >= 12.0 ? 2 : 1);
  const long long key = (long long)SHm | ((long long)SHj << 16) | ((long long)LR << 32);
  if (!h->gRef || h->gRef_key != key) {
    if ((s = build_refine_graph(h, SHm, SHj, LR)) != GABP_OK) return s;
    h->gRef_key = key;
  }
  RefineParams p;
  p.tol = tol;
  p.inner_tol = h->opt.inner_tol;
  p.prec_thr = std::ldexp(1.0, -h->opt.prec_stop_log2);
  p.max_refine = h->opt.max_refine;
  p.max_iter = max_iter;
  p.inner_max = h->opt.inner_max_iter;
  p.prec_cap = kPrecMaxRounds;
  p.joint = run_joint ? 1 : 0;
  GABP_CUDA(cudaMemcpyAsync(w.Bd, B, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, h->stream));
  k_ref_setup<<<1, 1, 0, h->stream>>>(w.rc, p);
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaGraphLaunch(h->gRef, h->stream));
  GABP_CUDA(cudaMemcpyAsync(X, w.X, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, h->stream));
  GABP_CUDA(cudaMemcpyAsync(w.rc_host, w.rc, sizeof(RefineCtl), cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  const RefineCtl r = *w.rc_host;
  h->prof.launches += 3 + (int64_t)r.launches;  // k_ref_setup, the first residual and decision, the loop
  if (run_joint) {
    if (r.prec_round >= 0) {
      w.prec_round = r.prec_round;
      w.coef_ready = true;
    } else if (r.status != GABP_BREAKDOWN && r.status != GABP_DIVERGED) {
      // stopped before any inner solve (b = 0): the precision state is still provided
      if ((s = precision_phase32(h, nullptr)) != GABP_OK) return s;
    }
  }
  h->stats.rounds += r.total_inner;
  h->stats.refine_steps = r.steps;
  if (iters) *iters = r.total_inner;
  if (relres) *relres = r.bb > 0.0 ? sqrt(r.rr / r.bb) : 0.0;
  return (gabp_status)r.status;
}

gabp_status solve32_refine(gabp_handle h, int R, const double *B, double *X, int64_t ld, double tol,
                           int max_iter, const double *gamma_diag, int *iters, double *relres) {
  NvtxRange nvtx_("gabp fp32 messages + fp64 refinement");
  if (R != 1) return GABP_ERR_INVALID;  // batched path: gabp_solve_batched
  (void)ld;
  gabp_status s = ensure_w32(h, 1);
  if (s != GABP_OK) return s;
  Work32 &w = h->w32;
  Graph &g = h->g;
  h->stats.rounds = 0;
  h->stats.edge_updates = -1;
  h->stats.refine_steps = 0;
  const bool serial = h->opt.schedule == 1 && !gamma_diag;
  if (h->opt.device_loop && h->opt.graphs && !gamma_diag && !h->opt.profile && h->stream && !serial)
    return solve32_device_loop(h, B, X, tol, max_iter, iters, relres);
  // the precision state is cached per handle when no loading is applied; when it
  // has to be computed, it is either computed first (precision-only rounds) or
  // together with the first inner solve (joint rounds, overlap_precision)
  bool joint = false;
  if (!w.coef_ready || gamma_diag || !h->opt.reuse_precisions) {
    w.coef_ready = false;
    joint = h->opt.overlap_precision != 0 && !serial;
    if (!joint) {
      if ((s = precision_phase32(h, gamma_diag)) != GABP_OK) return s;
      if (gamma_diag) w.coef_ready = false;  // do not reuse a loaded state for a plain solve
    }
  }
  if (serial && (s = serial_freeze32(h, w.CF, w.invP)) != GABP_OK) return s;  // coefficients in the serial order
  if (!serial && (s = autotune32(h, K32_MEAN)) != GABP_OK) return s;
  const int SH = shape32(h, K32_MEAN);
  // FP64 residual: narrow sub-warps (its per-row epilogue is FP64)
  const int LR = h->opt.lanes ? h->opt.lanes : (g.avg_deg >= 12.0 ? 2 : 1);
  int nbr = 1;
  GABP_DISPATCH_L(LR, nbr = blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, k64_residual<LL>)));
  GABP_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * g.n, h->stream));
  GABP_CUDA(cudaMemsetAsync(w.ctlR, 0, sizeof(DevCtl), h->stream));
  GABP_DISPATCH_L(LR, (k64_residual<LL><<<nbr, kBlock, 0, h->stream>>>(g.n, g.rowptr, g.col, g.val, B, X, w.rhs32,
                                                                          w.NH[0], w.ctlR, h->partials, 1, nullptr,
                                                                          1)));
  h->prof.launches += 1;
  GABP_CUDA(cudaGetLastError());
  DevCtl cr;
  GABP_CUDA(cudaMemcpyAsync(&cr, w.ctlR, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  const double bb = cr.bb;
  double rr = cr.rr;
  int total_inner = 0;
  gabp_status result = GABP_NOT_CONVERGED;
  if (bb == 0.0) {
    // x = 0; the precision state is still made available (marginal precisions)
    if (joint && (s = precision_phase32(h, gamma_diag)) != GABP_OK) return s;
    if (gamma_diag) w.coef_ready = false;
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return GABP_OK;
  }
  Args32 a = args32(h);
  const size_t E = (size_t)(g.E > 0 ? g.E : 1);
  const double itol = h->opt.inner_tol;
  for (int step = 0; step < h->opt.max_refine; ++step) {
    if (rr <= tol * tol * bb) { result = GABP_OK; break; }
    if (total_inner >= max_iter) break;
    // inner FP32 GaBP on A d = r (messages from zero, Algorithm 1 step 1); the
    // first one may start with the joint rounds, which leave round T's mean state
    const int cap = std::min(h->opt.inner_max_iter, std::max(1, max_iter - total_inner));
    const double it_tol = inner_target(itol, tol, bb, rr);
    if (serial) {  // serial frozen-coefficient sweeps (serial.cu)
      int sweeps = 0, ist = 0;
      if ((s = serial_inner32(h, w.rhs32, cap, it_tol, &sweeps, &ist)) != GABP_OK) return s;
      total_inner += sweeps;
      h->stats.rounds += sweeps;
      if (ist == GABP_DIVERGED) { result = GABP_DIVERGED; break; }
      prof_begin(h);
      if ((s = serial_update32(h, X)) != GABP_OK) return s;
      GABP_DISPATCH_L(LR, (k64_residual<LL><<<nbr, kBlock, 0, h->stream>>>(g.n, g.rowptr, g.col, g.val, B, X, w.rhs32,
                                                                              w.NH[0], w.ctlR, h->partials, 0)));
      prof_end(h);
      h->prof.launches += 2;
      GABP_CUDA(cudaGetLastError());
      GABP_CUDA(cudaMemcpyAsync(&cr, w.ctlR, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
      GABP_CUDA(cudaStreamSynchronize(h->stream));
      prof_collect(h, PH_REFINE64, 1);
      h->stats.refine_steps = step + 1;
      if (!std::isfinite(cr.rr)) { result = GABP_DIVERGED; rr = cr.rr; break; }
      rr = cr.rr;
      continue;
    }
    int T = 0;
    if (step == 0 && joint) {
      if ((s = joint_phase32(h, gamma_diag, cap, &T)) != GABP_OK) return s;
      // freeze at T fused with the first frozen-coefficient round T + 1
      k_ctl_reset<<<1, 1, 0, h->stream>>>(h->ctl, cap, it_tol * it_tol, T);
      h->prof.launches += 1;
      if ((s = freeze32(h, T)) != GABP_OK) return s;
      if (gamma_diag) w.coef_ready = false;  // do not reuse a loaded state for a plain solve
    } else {
      GABP_CUDA(cudaMemsetAsync(w.H[0], 0, sizeof(float) * E, h->stream));
    }
    int result_round = T;
    if (T < cap) {
      if (T == 0) {
        k_ctl_reset<<<1, 1, 0, h->stream>>>(h->ctl, cap, it_tol * it_tol, 0);
        h->prof.launches += 1;
      }
      GABP_CUDA(cudaGetLastError());
      with_shape(SH, [&](auto Lc, auto Uc) {
        constexpr int LL = decltype(Lc)::value, UU = decltype(Uc)::value;
        s = run_rounds(h, &h->gH32, &h->gH32_L, SH, [&] {
          launch_mean<LL, UU>(h, a, h->stream);
        }, cap - T, PH_MEAN32, T > 0 ? T + 1 : 0);
      });
      if (s != GABP_OK) return s;
      const DevCtl c = *h->ctl_host;
      result_round = c.result_round;
      if (c.status == GABP_DIVERGED) {
        total_inner += c.round;
        h->stats.rounds += c.round;
        result = GABP_DIVERGED;
        break;
      }
    }
    total_inner += result_round;
    h->stats.rounds += result_round;
    float *hT = result_round % 3 == 0 ? w.NH[0] : (result_round % 3 == 1 ? w.NH[1] : w.NH[2]);
    prof_begin(h);
    k64_update<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, X, hT, w.invP);
    GABP_DISPATCH_L(LR, (k64_residual<LL><<<nbr, kBlock, 0, h->stream>>>(g.n, g.rowptr, g.col, g.val, B, X, w.rhs32,
                                                                            w.NH[0], w.ctlR, h->partials, 0)));
    prof_end(h);
    h->prof.launches += 2;
    GABP_CUDA(cudaGetLastError());
    GABP_CUDA(cudaMemcpyAsync(&cr, w.ctlR, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
    GABP_CUDA(cudaStreamSynchronize(h->stream));
    prof_collect(h, PH_REFINE64, 1);
    h->stats.refine_steps = step + 1;
    if (!std::isfinite(cr.rr)) { result = GABP_DIVERGED; rr = cr.rr; break; }
    rr = cr.rr;
  }
  if (result != GABP_DIVERGED && rr <= tol * tol * bb) result = GABP_OK;
  if (iters) *iters = total_inner;
  if (relres) *relres = sqrt(rr / bb);
  return result;
}

}  // namespace gabp
