// multigrid.cu -- many independent systems in ONE persistent cooperative launch,
// every system advancing through its own state machine while the whole grid
// sweeps the rows of all systems still running.
//
// Per global round, every active system makes one step of its own solve:
//   PREC   one FP32 precision round (recompute form of Algorithm 2),
//   COEF   freeze c_in, c_out, 1/P~ and set x = 0,
//   RESID  r = b - A x in FP64, FP32 copy as the inner right-hand side,
//   INNER  one FP32 mean round of the inner solve of A d = r,
//   UPDATE x += d (FP64),
// and its row sums (max change of the precisions, the inner ||dx||^2 and
// ||x||^2, the outer ||r||^2) are gathered per system.  Each round ends with
// ONE grid barrier: the last block to arrive takes every system's decision
// (stationary precisions, inner tolerance reached -- with the adaptive target
// of solve32.cu -- outer tolerance reached, breakdown, divergence, caps) and
// then releases the others.  Systems therefore converge independently, as if
// solved one by one, while each round streams the rows of all running systems.
// L lanes work on one row (coalesced slot loads), U slots per lane have their
// loads issued together.
//
// The barrier spins on a generation counter with a clock-bounded wait: all
// blocks are co-resident (cooperative launch), so it always completes; if it
// ever did not within ~2 s, the kernel records GABP_TIMEOUT and returns.
#include "gabp_internal.cuh"
#include "devutil.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace gabp {

namespace {

enum : int { PH_PREC = 0, PH_COEF = 1, PH_RESID = 2, PH_INNER = 3, PH_UPDATE = 4, PH_DONE = 5 };
constexpr int kGPrecCap = 300;               // precision-round cap per system
constexpr int kGChunkMax = 8;                // warp steps per chunk of contiguous rows (at most)
constexpr long long kBarrierLimit = 4000000000LL;  // clock cycles (~2 s) before a barrier gives up

struct SysState {
  int phase, t, stable, Tp, Tm, steps, inner_total, status;
  double bb, rr, itol, pad;
};

struct GridArgs {
  int n, nsys;
  int chunk;                        // warp steps (sliced kernel: slices) per chunk, enough chunks per warp
                                    // to balance the round
  int ns;                           // sliced kernel: slices, their rows, first slots and systems
  const int *__restrict__ srow;
  const int *__restrict__ sp;
  const int *__restrict__ ssys;
  const int *__restrict__ sys_of;   // row -> system
  const int *__restrict__ rp;
  const int *__restrict__ ci;
  const float *__restrict__ av;
  const float *__restrict__ ad;
  const int *__restrict__ rowptr;
  const int *__restrict__ col;
  const double *__restrict__ val;
  float *MP0, *MP1, *NP0, *NP1, *NP2;
  float2 *CF;
  float *invP;
  float *H0, *H1, *NH0, *NH1, *NH2;
  float *rhs;
  const double *b;
  double *x;
  SysState *st;        // [nsys]
  double *acc;         // [nsys][4] per-round sums: 0 bad / rr / dxx, 1 max-rel / xx
  unsigned int *bar;   // [0] arrival count, [1] generation
  int *active;         // running-system count of the round
  int *err;            // nonzero once a barrier gave up
  double tol, inner_tol, prec_thr;
  int inner_max, max_refine, max_iter, max_rounds;
};

__device__ __forceinline__ float *ring(float *a, float *b, float *c, int t) {
  const int m = t % 3;
  return m == 0 ? a : (m == 1 ? b : c);
}

// Per-warp running sums of one system (slot 0: sum; slot 1: sum, or max for
// the precision rounds' relative change), flushed to the system's accumulators
// in global memory only when the warp meets another system or ends its pass:
// a warp reads contiguous chunks of rows, so most rows fold in registers and a
// system's accumulator sees a few atomics per chunk, not one per row.  A NaN in
// a max survives (it must not read as "stationary"); 0 is neutral for the max
// too, the values being >= 0 or NaN.
struct WarpAcc {
  int s = -1;
  bool max1 = false;
  double r0 = 0.0, r1 = 0.0;

  __device__ __forceinline__ void flush(double *acc) {
    if (s < 0) return;  // warp-uniform
    double a0 = r0, a1 = r1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      const double b1 = __shfl_xor_sync(0xffffffffu, a1, o);
      a1 = max1 ? nan_max(a1, b1) : a1 + b1;
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(acc + 4 * s, a0);
      if (max1)
        atomicMax(reinterpret_cast<unsigned long long *>(acc + 4 * s + 1), (unsigned long long)__double_as_longlong(a1));
      else
        atomicAdd(acc + 4 * s + 1, a1);
    }
    s = -1;
    r0 = r1 = 0.0;
  }

  // one row's values (lanes with has = false contribute nothing); all lanes call
  __device__ __forceinline__ void add(double *acc, int sys, double v0, double v1, bool mx, bool has) {
    const unsigned with = __ballot_sync(0xffffffffu, has);
    if (!with) return;
    const int src = __ffs(with) - 1;
    const int s0 = __shfl_sync(0xffffffffu, sys, src);
    if (__all_sync(0xffffffffu, !has || sys == s0)) {
      if (s0 != s) {
        flush(acc);
        s = s0;
        max1 = __shfl_sync(0xffffffffu, mx, src);
      }
      if (has) {
        r0 += v0;
        r1 = max1 ? nan_max(r1, v1) : r1 + v1;
      }
    } else if (has) {  // rows of several systems in this warp step: direct atomics
      atomicAdd(acc + 4 * sys, v0);
      if (mx)
        atomicMax(reinterpret_cast<unsigned long long *>(acc + 4 * sys + 1), (unsigned long long)__double_as_longlong(v1));
      else
        atomicAdd(acc + 4 * sys + 1, v1);
    }
  }
};

// Per-lane running sums of one system for the sliced kernel, whose slices each belong
// to one system (the system is warp-uniform): the precision and inner rounds' row
// values fold in FP32 registers (sum, and max for the precision rounds' relative
// change; a NaN survives the max) and are reduced across the warp in FP32, lane 0
// converting the two totals to FP64 for the system's accumulators; only the FP64
// residual is summed and reduced in FP64.  A warp flushes whenever it meets another
// system, which with short chunks is about once per slice, so the flush keeps off
// the FP64 pipe.
struct SliceAcc {
  int s = -1;
  bool max1 = false, dbl = false;
  float f0 = 0.f, f1 = 0.f;
  double d0 = 0.0;

  __device__ __forceinline__ void flush(double *acc) {
    if (s < 0) return;  // warp-uniform
    if (dbl) {
      double a0 = d0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      if ((threadIdx.x & 31) == 0) atomicAdd(acc + 4 * s, a0);
    } else {
      float a0 = f0, a1 = f1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        const float b1 = __shfl_xor_sync(0xffffffffu, a1, o);
        a1 = max1 ? nan_max(a1, b1) : a1 + b1;
      }
      if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc + 4 * s, (double)a0);
        if (max1)  // values >= 0 or NaN: the bit patterns order as the values
          atomicMax(reinterpret_cast<unsigned long long *>(acc + 4 * s + 1),
                    (unsigned long long)__double_as_longlong((double)a1));
        else
          atomicAdd(acc + 4 * s + 1, (double)a1);
      }
    }
    s = -1;
    f0 = f1 = 0.f;
    d0 = 0.0;
  }
  // all lanes call it with the same sys and phase
  __device__ __forceinline__ void to(double *acc, int sys, int ph) {
    if (sys != s) {
      flush(acc);
      s = sys;
      max1 = ph == PH_PREC;
      dbl = ph == PH_RESID;
    }
  }
};

// A system's state as last written by the deciding block (possibly on another
// SM): read through L2.
__device__ __forceinline__ SysState load_state(const SysState *p) {
  SysState S;
  const int4 *q = reinterpret_cast<const int4 *>(p);
  int4 *d = reinterpret_cast<int4 *>(&S);
#pragma unroll
  for (int j = 0; j < (int)(sizeof(SysState) / sizeof(int4)); ++j) d[j] = __ldcg(q + j);
  return S;
}

// One system's decision after a round (run by the deciding block).  Returns 1
// while the system is still running.
__device__ int decide(const GridArgs &a, int s) {
  SysState S = load_state(a.st + s);
  double *ac = a.acc + 4 * s;
  const double v0 = __ldcg(ac), v1 = __ldcg(ac + 1);
  ac[0] = 0.0;
  ac[1] = 0.0;
  switch (S.phase) {
    case PH_PREC: {
      S.stable = (v1 <= a.prec_thr) ? S.stable + 1 : 0;  // a NaN is not stationary
      if (v0 > 0.0) { S.status = GABP_BREAKDOWN; S.phase = PH_DONE; S.Tp = S.t; }
      else if (!(v1 <= 1e30)) { S.status = GABP_DIVERGED; S.phase = PH_DONE; S.Tp = S.t; }
      else if (S.stable >= 2 || S.t >= kGPrecCap) { S.Tp = S.t; S.phase = PH_COEF; }
      else S.t += 1;
      break;
    }
    case PH_COEF: S.phase = PH_RESID; break;
    case PH_RESID: {
      S.rr = v0;
      if (S.steps == 0) S.bb = v0;
      if (S.bb == 0.0 || S.rr <= a.tol * a.tol * S.bb) { S.status = GABP_OK; S.phase = PH_DONE; }
      else if (!isfinite(S.rr)) { S.status = GABP_DIVERGED; S.phase = PH_DONE; }
      else if (S.steps >= a.max_refine || S.inner_total >= a.max_iter) { S.status = GABP_NOT_CONVERGED; S.phase = PH_DONE; }
      else {
        const double need = 0.1 * a.tol * sqrt(S.bb / S.rr);
        S.itol = fmin(a.inner_tol, fmax(1e-6, need));
        S.phase = PH_INNER;
        S.t = 1;
      }
      break;
    }
    case PH_INNER: {
      const int cap = min(a.inner_max, max(1, a.max_iter - S.inner_total));
      if (!isfinite(v0) || !isfinite(v1)) { S.status = GABP_DIVERGED; S.phase = PH_DONE; S.inner_total += S.t; }
      else if ((S.t >= 2 && v0 <= S.itol * S.itol * v1) || S.t >= cap) {
        S.Tm = S.t;
        S.inner_total += S.t;
        S.phase = PH_UPDATE;
      } else S.t += 1;
      break;
    }
    case PH_UPDATE: S.steps += 1; S.phase = PH_RESID; break;
    default: return 0;
  }
  a.st[s] = S;
  return S.phase != PH_DONE;
}

// End of a round: bounded grid barrier whose last arriving block takes all
// decisions before it releases the others.  Returns the number of systems still
// running, or -1 if a wait gave up.
__device__ int round_end(const GridArgs &a) {
  __shared__ int s_last, s_act;
  __shared__ unsigned s_gen;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = *(volatile unsigned *)(a.bar + 1);
    __threadfence();
    s_last = atomicAdd(a.bar, 1u) == gridDim.x - 1;
    s_gen = g;
    s_act = 0;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    int mine = 0;
    for (int s = threadIdx.x; s < a.nsys; s += blockDim.x) mine += decide(a, s);
    if (mine) atomicAdd(&s_act, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
      *(volatile int *)a.active = s_act;
      a.bar[0] = 0;
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    }
  } else if (threadIdx.x == 0) {
    volatile unsigned *gen = a.bar + 1;
    const long long t0 = clock64();
    int ok = 1;
    while (*gen == s_gen) {
      if (*(volatile int *)a.err || clock64() - t0 > kBarrierLimit) { ok = 0; break; }
      __nanosleep(64);
    }
    if (!ok) atomicExch(a.err, 1);
    __threadfence();
    s_act = ok ? *(volatile int *)a.active : -1;
  }
  __syncthreads();
  return s_act;
}

template <int L, int U>
__global__ void __launch_bounds__(kBlock, U >= 4 ? 3 : (U == 2 ? 4 : 5)) kg_solve(GridArgs a) {
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  const int CR = RPW * a.chunk;  // rows per chunk
  const int nchunks = (a.n + CR - 1) / CR;
  for (int round = 0; round < a.max_rounds; ++round) {
    WarpAcc wacc;
    int sc = -1, phc = PH_DONE, tc = 0, Tc = 0;  // this lane's cached system state (fixed within a round)
    // warp-uniform loops: every lane of a warp runs every iteration
    for (int chunk = warp; chunk < nchunks; chunk += nwarps)
    for (int base = chunk * CR; base < min(a.n, (chunk + 1) * CR); base += RPW) {
      const int i = base + sw;
      int s = -1, ph = PH_DONE, t = 0, T = 0;
      if (i < a.n) {
        s = a.sys_of[i];
        if (s != sc) {
          const SysState S = load_state(a.st + s);
          sc = s;
          phc = S.phase;
          tc = S.t;
          Tc = S.phase == PH_COEF ? S.Tp : S.Tm;
        }
        ph = phc;
        t = tc;
        T = Tc;
      }
      // ---------------------------------------------------------- edge part, L lanes per row
      float facc = 0.f, frel = 0.f;
      float rhs_i = 0.f, ip_i = 0.f, hprev_i = 0.f;  // row values of an inner round
      double dacc = 0.0;
      int bad = 0;
      if (ph == PH_PREC) {
        float *Mc = (t & 1) ? a.MP1 : a.MP0;
        const float *Mo = (t & 1) ? a.MP0 : a.MP1;
        const float *Pm1 = ring(a.NP0, a.NP1, a.NP2, t + 2);
        const float Pi2 = t >= 2 ? ring(a.NP0, a.NP1, a.NP2, t + 1)[i] : 0.f;
        const int e1 = a.rp[i + 1];
        for (int eb = a.rp[i] + sl; eb < e1; eb += L * U) {
          int k[U];
          float A[U], Ps[U], Pp[U], Pk[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int e = eb + u * L;
            if (e < e1) { k[u] = a.ci[e]; A[u] = a.av[e]; Ps[u] = Mc[e]; Pp[u] = Mo[e]; }
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (eb + u * L < e1) Pk[u] = __ldcg(Pm1 + k[u]);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int e = eb + u * L;
            if (e < e1) {
              // fast FP32 division (about 2 ulp), as in the single-system precision rounds: the
              // precision state only has to be FP32-accurate, the FP64 refinement absorbs the rest
              const float A2 = A[u] * A[u];
              float Pout = 0.f;
              if (t >= 2) {
                const float d1 = Pi2 - Ps[u];
                bad |= (d1 == 0.f);
                Pout = -__fdividef(A2, d1);
              }
              const float d2 = Pk[u] - Pout;
              bad |= (d2 == 0.f);
              const float Pn = -__fdividef(A2, d2);
              Mc[e] = Pn;
              facc += Pn;
              const float dP = fabsf(Pn - Pp[u]);
              frel = nan_max(frel, dP == 0.f ? 0.f : __fdividef(dP, fabsf(Pn)));
            }
          }
        }
      } else if (ph == PH_COEF) {
        const float *Ms = (T & 1) ? a.MP1 : a.MP0;
        const float *PT = ring(a.NP0, a.NP1, a.NP2, T);
        const float Pi = PT[i];
        for (int e = a.rp[i] + sl; e < a.rp[i + 1]; e += L) {
          const float A = a.av[e];
          const float cout = -A / (Pi - Ms[e]);
          const float cin = -A / (__ldcg(PT + a.ci[e]) - cout * A);
          a.CF[e] = make_float2(cin, cout);
        }
      } else if (ph == PH_RESID) {
        for (int p = a.rowptr[i] + sl; p < a.rowptr[i + 1]; p += L) dacc = fma(a.val[p], __ldcg(a.x + a.col[p]), dacc);
        for (int e = a.rp[i] + sl; e < a.rp[i + 1]; e += L) a.H0[e] = 0.f;
      } else if (ph == PH_INNER) {
        float *Hc = (t & 1) ? a.H1 : a.H0;
        const float *Hm1 = ring(a.NH0, a.NH1, a.NH2, t + 2);
        const float hi2 = t >= 2 ? ring(a.NH0, a.NH1, a.NH2, t + 1)[i] : 0.f;
        // the row's own values are requested before its slots (used by the node part below)
        rhs_i = a.rhs[i];
        ip_i = a.invP[i];
        hprev_i = Hm1[i];
        const int e1 = a.rp[i + 1];
        for (int eb = a.rp[i] + sl; eb < e1; eb += L * U) {
          int k[U];
          float2 cf[U];
          float hs[U], hk[U];
          // slot arrays belong to the row (written only by its own lanes): streamed, evict-first
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int e = eb + u * L;
            if (e < e1) { k[u] = __ldcs(a.ci + e); cf[u] = __ldcs(a.CF + e); hs[u] = __ldcs(Hc + e); }
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (eb + u * L < e1) hk[u] = __ldcg(Hm1 + k[u]);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int e = eb + u * L;
            if (e < e1) {
              const float hout = t >= 2 ? cf[u].y * (hi2 - hs[u]) : 0.f;
              const float hn = cf[u].x * (hk[u] - hout);
              __stcs(Hc + e, hn);
              facc += hn;
            }
          }
        }
      }
      // ---------------------------------------------------------- row sums over the L lanes
      facc = sub_sum<L>(facc);
      dacc = sub_sum<L>(dacc);
      bad = sub_sum<L>(bad);
#pragma unroll
      for (int o = L / 2; o > 0; o >>= 1) frel = nan_max(frel, __shfl_xor_sync(0xffffffffu, frel, o, L));
      // ---------------------------------------------------------- node part, one lane per row
      double c0 = 0.0, c1 = 0.0;
      bool has = false;
      if (sl == 0 && ph != PH_DONE) {
        if (ph == PH_PREC) {
          const float P = a.ad[i] + facc;
          bad |= (P == 0.f);
          ring(a.NP0, a.NP1, a.NP2, t)[i] = P;
          c0 = (double)bad;
          c1 = (double)frel;
          has = true;
        } else if (ph == PH_COEF) {
          a.invP[i] = 1.f / ring(a.NP0, a.NP1, a.NP2, T)[i];
          a.x[i] = 0.0;
        } else if (ph == PH_RESID) {
          const double r = a.b[i] - dacc;
          a.rhs[i] = (float)r;
          a.NH0[i] = (float)r;
          c0 = r * r;
          has = true;
        } else if (ph == PH_INNER) {
          const float hnew = rhs_i + facc;
          ring(a.NH0, a.NH1, a.NH2, t)[i] = hnew;
          const float xi = hnew * ip_i, dx = (hnew - hprev_i) * ip_i;
          c0 = (double)(dx * dx);
          c1 = (double)(xi * xi);
          has = true;
        } else if (ph == PH_UPDATE) {
          a.x[i] += (double)(ring(a.NH0, a.NH1, a.NH2, T)[i] * a.invP[i]);
        }
      }
      wacc.add(a.acc, s, c0, c1, ph == PH_PREC, has);
    }
    wacc.flush(a.acc);
    const int act = round_end(a);
    if (act <= 0) return;
  }
}

// The same global rounds on the sliced layout (GSell): a warp per 32-row slice, a lane
// per row, slot j of the slice's rows one contiguous line (ci, av and the message and
// coefficient arrays are the layout's); U slots of a row have their loads issued
// together.  A slice belongs to one system, so its phase is warp-uniform and the
// slices of finished systems are skipped.  Per slot the arithmetic is kg_solve's
// with one lane per row; the FP64 residual reads the input CSR row by row.
template <int U>
__global__ void __launch_bounds__(kBlock, U >= 4 ? 3 : 4) kgs_solve(GridArgs a) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  const int nchunks = (a.ns + a.chunk - 1) / a.chunk;
  for (int round = 0; round < a.max_rounds; ++round) {
    SliceAcc sacc;
    int sc = -1, ph = PH_DONE, t = 0, T = 0;  // the current slice's system state (fixed within a round)
    for (int chunk = warp; chunk < nchunks; chunk += nwarps)
    for (int sl = chunk * a.chunk; sl < min(a.ns, (chunk + 1) * a.chunk); ++sl) {
      const int s = a.ssys[sl];
      if (s != sc) {
        const SysState S = load_state(a.st + s);
        sc = s;
        ph = S.phase;
        t = S.t;
        T = S.phase == PH_COEF ? S.Tp : S.Tm;
      }
      if (ph == PH_DONE) continue;  // warp-uniform
      const int i = a.srow[sl * 32 + lane];
      const int q0 = a.sp[sl];
      const int p0 = q0 + lane, wd = (a.sp[sl + 1] - q0) >> 5;
      float facc = 0.f, frel = 0.f;
      float rhs_i = 0.f, ip_i = 0.f, hprev_i = 0.f;
      double dacc = 0.0;
      int bad = 0;
      if (ph == PH_PREC) {
        float *Mc = (t & 1) ? a.MP1 : a.MP0;
        const float *Mo = (t & 1) ? a.MP0 : a.MP1;
        const float *Pm1 = ring(a.NP0, a.NP1, a.NP2, t + 2);
        const float Pi2 = (t >= 2 && i >= 0) ? ring(a.NP0, a.NP1, a.NP2, t + 1)[i] : 0.f;
        for (int j = 0; j < wd; j += U) {
          int k[U];
          float A[U], Ps[U], Pp[U], Pk[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int pos = p0 + 32 * (j + u);
            k[u] = j + u < wd ? __ldcs(a.ci + pos) : -1;
            if (k[u] >= 0) { A[u] = __ldcs(a.av + pos); Ps[u] = __ldcs(Mc + pos); Pp[u] = __ldcs(Mo + pos); }
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (k[u] >= 0) Pk[u] = __ldcg(Pm1 + k[u]);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (k[u] < 0) continue;
            const float A2 = A[u] * A[u];
            float Pout = 0.f;
            if (t >= 2) {
              const float d1 = Pi2 - Ps[u];
              bad |= (d1 == 0.f);
              Pout = -__fdividef(A2, d1);
            }
            const float d2 = Pk[u] - Pout;
            bad |= (d2 == 0.f);
            const float Pn = -__fdividef(A2, d2);
            __stcs(Mc + p0 + 32 * (j + u), Pn);
            facc += Pn;
            const float dP = fabsf(Pn - Pp[u]);
            frel = nan_max(frel, dP == 0.f ? 0.f : __fdividef(dP, fabsf(Pn)));
          }
        }
      } else if (ph == PH_COEF) {
        if (i >= 0) {
          const float *Ms = (T & 1) ? a.MP1 : a.MP0;
          const float *PT = ring(a.NP0, a.NP1, a.NP2, T);
          const float Pi = PT[i];
          for (int j = 0; j < wd; ++j) {
            const int pos = p0 + 32 * j;
            const int k = __ldcs(a.ci + pos);
            if (k < 0) break;  // a row's padding slots follow its real ones
            const float A = __ldcs(a.av + pos);
            const float cout = -A / (Pi - Ms[pos]);
            const float cin = -A / (__ldcg(PT + k) - cout * A);
            a.CF[pos] = make_float2(cin, cout);
          }
        }
      } else if (ph == PH_RESID) {
        if (i >= 0)
          for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) dacc = fma(a.val[p], __ldcg(a.x + a.col[p]), dacc);
        for (int j = 0; j < wd; ++j) a.H0[p0 + 32 * j] = 0.f;
      } else if (ph == PH_INNER) {
        float *Hc = (t & 1) ? a.H1 : a.H0;
        const float *Hm1 = ring(a.NH0, a.NH1, a.NH2, t + 2);
        float hi2 = 0.f;
        if (i >= 0) {  // the row's own values are requested before its slots
          hi2 = t >= 2 ? ring(a.NH0, a.NH1, a.NH2, t + 1)[i] : 0.f;
          rhs_i = a.rhs[i];
          ip_i = a.invP[i];
          hprev_i = Hm1[i];
        }
        for (int j = 0; j < wd; j += U) {
          int k[U];
          float2 cf[U];
          float hs[U], hk[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int pos = p0 + 32 * (j + u);
            k[u] = j + u < wd ? __ldcs(a.ci + pos) : -1;
            if (k[u] >= 0) { cf[u] = __ldcs(a.CF + pos); hs[u] = __ldcs(Hc + pos); }
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (k[u] >= 0) hk[u] = __ldcg(Hm1 + k[u]);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (k[u] < 0) continue;
            const float hout = t >= 2 ? cf[u].y * (hi2 - hs[u]) : 0.f;
            const float hn = cf[u].x * (hk[u] - hout);
            __stcs(Hc + p0 + 32 * (j + u), hn);
            facc += hn;
          }
        }
      }
      // ---------------------------------------------------------- node part, one lane per row
      sacc.to(a.acc, s, ph);
      if (i >= 0) {
        if (ph == PH_PREC) {
          const float P = a.ad[i] + facc;
          bad |= (P == 0.f);
          ring(a.NP0, a.NP1, a.NP2, t)[i] = P;
          sacc.f0 += (float)bad;
          sacc.f1 = nan_max(sacc.f1, frel);
        } else if (ph == PH_COEF) {
          a.invP[i] = 1.f / ring(a.NP0, a.NP1, a.NP2, T)[i];
          a.x[i] = 0.0;
        } else if (ph == PH_RESID) {
          const double r = a.b[i] - dacc;
          a.rhs[i] = (float)r;
          a.NH0[i] = (float)r;
          sacc.d0 = fma(r, r, sacc.d0);
        } else if (ph == PH_INNER) {
          const float hnew = rhs_i + facc;
          ring(a.NH0, a.NH1, a.NH2, t)[i] = hnew;
          const float xi = hnew * ip_i, dx = (hnew - hprev_i) * ip_i;
          sacc.f0 = fmaf(dx, dx, sacc.f0);
          sacc.f1 = fmaf(xi, xi, sacc.f1);
        } else if (ph == PH_UPDATE) {
          a.x[i] += (double)(ring(a.NH0, a.NH1, a.NH2, T)[i] * a.invP[i]);
        }
      }
    }
    sacc.flush(a.acc);
    const int act = round_end(a);
    if (act <= 0) return;
  }
}

// Slot arrays of the sliced layout from the off-diagonal CSR (one thread per slice lane).
__global__ void kgs_fill(int nq, const int *__restrict__ srow, const int *__restrict__ sp,
                         const int *__restrict__ rp, const int *__restrict__ ci, const float *__restrict__ av,
                         int *sci, float *sav) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int sl = q >> 5, lane = q & 31, i = srow[q];
  const int p0 = sp[sl] + lane, wd = (sp[sl + 1] - sp[sl]) >> 5;
  const int e0 = i >= 0 ? rp[i] : 0, deg = i >= 0 ? rp[i + 1] - e0 : 0;
  for (int j = 0; j < wd; ++j) {
    const int pos = p0 + 32 * j;
    sci[pos] = j < deg ? ci[e0 + j] : -1;
    sav[pos] = j < deg ? av[e0 + j] : 0.f;
  }
}

__global__ void kg_init(int nsys, SysState *st, double *acc, const int *__restrict__ offsets, int *sys_of) {
  const int s = blockIdx.x;
  if (s >= nsys) return;
  if (threadIdx.x == 0) {
    SysState S = {};
    S.phase = PH_PREC;
    S.t = 1;
    S.status = GABP_NOT_CONVERGED;
    st[s] = S;
    for (int j = 0; j < 4; ++j) acc[4 * s + j] = 0.0;
  }
  for (int i = offsets[s] + threadIdx.x; i < offsets[s + 1]; i += blockDim.x) sys_of[i] = s;
}

// round-0 precision state of every row: P~ = A_ii (FP32), zero messages, x = 0
__global__ void kg_rows_init(int n, const int *__restrict__ rp, const double *__restrict__ ad, float *ad32,
                             float *NP0, float *MP0, float *MP1, double *x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float d = (float)ad[i];
    ad32[i] = d;
    NP0[i] = d;
    x[i] = 0.0;
    if (MP0)  // the CSR kernels' messages (the sliced layout's are cleared with a memset)
      for (int e = rp[i]; e < rp[i + 1]; ++e) { MP0[e] = 0.f; MP1[e] = 0.f; }
  }
}

// kernel for a shape code L | U << 8 (| kSliced for the sliced layout; unknown codes: (4, 2))
void (*grid_kernel(int code))(GridArgs) {
  switch (code) {
    case kGridShapes[9]: return kgs_solve<1>;
    case kGridShapes[10]: return kgs_solve<2>;
    case kGridShapes[11]: return kgs_solve<4>;
    case kGridShapes[0]: return kg_solve<1, 4>;
    case kGridShapes[1]: return kg_solve<2, 4>;
    case kGridShapes[3]: return kg_solve<4, 4>;
    case kGridShapes[4]: return kg_solve<8, 2>;
    case kGridShapes[5]: return kg_solve<1, 2>;
    case kGridShapes[6]: return kg_solve<2, 2>;
    case kGridShapes[7]: return kg_solve<1, 1>;
    case kGridShapes[8]: return kg_solve<2, 1>;
    default: return kg_solve<4, 2>;
  }
}

}  // namespace

void free_gsell(gabp_handle h) {
  GSell *L = h->gsl;
  if (!L) return;
  cudaFree(L->srow); cudaFree(L->sp); cudaFree(L->ssys); cudaFree(L->sci); cudaFree(L->sav);
  cudaFree(L->MP[0]); cudaFree(L->MP[1]); cudaFree(L->H[0]); cudaFree(L->H[1]); cudaFree(L->CF);
  delete L;
  h->gsl = nullptr;
}

// The sliced layout for these offsets (rebuilt when they differ from the cached one),
// its slot values refreshed after gabp_set_values.
static gabp_status ensure_gsell(gabp_handle h, int nsys, const int *off) {
  Graph &g = h->g;
  GSell *L = h->gsl;
  if (!(L && (int)L->off.size() == nsys + 1 && std::equal(L->off.begin(), L->off.end(), off))) {
    free_gsell(h);
    L = h->gsl = new GSell();
    std::vector<int> rp(g.n + 1);
    GABP_CUDA(cudaMemcpyAsync(rp.data(), g.rp, sizeof(int) * (g.n + 1), cudaMemcpyDeviceToHost, h->stream));
    GABP_CUDA(cudaStreamSynchronize(h->stream));
    std::vector<int> srow, sp(1, 0), ssys, rows;
    long long slots = 0;
    for (int s = 0; s < nsys; ++s) {
      const int a0 = off[s], ns = off[s + 1] - off[s];
      rows.resize(ns);
      for (int r = 0; r < ns; ++r) rows[r] = a0 + r;
      for (int w0 = 0; w0 < ns; w0 += 4096)
        std::stable_sort(rows.begin() + w0, rows.begin() + std::min(ns, w0 + 4096),
                         [&](int x, int y) { return rp[x + 1] - rp[x] > rp[y + 1] - rp[y]; });
      for (int q = 0; q < ns; q += 32) {
        int wd = 0;
        for (int l = 0; l < 32; ++l) {
          const int r = q + l < ns ? rows[q + l] : -1;
          srow.push_back(r);
          if (r >= 0) wd = std::max(wd, rp[r + 1] - rp[r]);
        }
        slots += 32LL * wd;
        if (slots > 0x7fffffffLL) {
          set_last_error("gabp_solve_systems: the sliced layout would exceed 2^31 slots");
          free_gsell(h);
          return GABP_ERR_NOMEM;
        }
        sp.push_back((int)slots);
        ssys.push_back(s);
      }
    }
    L->ns = (int)ssys.size();
    L->Es = (int)slots;
    const size_t Ea = std::max<size_t>(1, (size_t)L->Es);
    GABP_CUDA(cudaMalloc(&L->srow, sizeof(int) * srow.size()));
    GABP_CUDA(cudaMalloc(&L->sp, sizeof(int) * sp.size()));
    GABP_CUDA(cudaMalloc(&L->ssys, sizeof(int) * ssys.size()));
    GABP_CUDA(cudaMalloc(&L->sci, sizeof(int) * Ea));
    GABP_CUDA(cudaMalloc(&L->sav, sizeof(float) * Ea));
    for (int c = 0; c < 2; ++c) {
      GABP_CUDA(cudaMalloc(&L->MP[c], sizeof(float) * Ea));
      GABP_CUDA(cudaMalloc(&L->H[c], sizeof(float) * Ea));
    }
    GABP_CUDA(cudaMalloc(&L->CF, sizeof(float2) * Ea));
    GABP_CUDA(cudaMemcpyAsync(L->srow, srow.data(), sizeof(int) * srow.size(), cudaMemcpyHostToDevice, h->stream));
    GABP_CUDA(cudaMemcpyAsync(L->sp, sp.data(), sizeof(int) * sp.size(), cudaMemcpyHostToDevice, h->stream));
    GABP_CUDA(cudaMemcpyAsync(L->ssys, ssys.data(), sizeof(int) * ssys.size(), cudaMemcpyHostToDevice, h->stream));
    GABP_CUDA(cudaStreamSynchronize(h->stream));  // the host vectors are released on return
    L->off.assign(off, off + nsys + 1);            // complete: reusable for these offsets
    L->vals_ok = false;
  }
  if (!L->vals_ok) {
    const int nq = 32 * L->ns;
    kgs_fill<<<(nq + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(nq, L->srow, L->sp, g.rp, g.ci, g.av32, L->sci,
                                                                   L->sav);
    GABP_CUDA(cudaGetLastError());
    L->vals_ok = true;
  }
  return GABP_OK;
}

gabp_status solve_systems_grid(gabp_handle h, int nsys, const int *d_off, const int *off_host, const double *b,
                               double *x, double tol, int max_iter, int *d_status, int *d_iters, int *d_refine,
                               double *d_relres, int shape, float *ms_out) {
  Graph &g = h->g;
  Work32 &w = h->w32;
  struct Free {
    std::vector<void *> p;
    ~Free() { for (void *q : p) cudaFree(q); }
  } fr;
  SysState *st = nullptr;
  double *acc = nullptr;
  int *sys_of = nullptr, *misc = nullptr;
  unsigned int *bar = nullptr;
  GABP_CUDA(cudaMalloc(&st, sizeof(SysState) * nsys));
  fr.p.push_back(st);
  GABP_CUDA(cudaMalloc(&acc, sizeof(double) * 4 * nsys));
  fr.p.push_back(acc);
  GABP_CUDA(cudaMalloc(&sys_of, sizeof(int) * g.n));
  fr.p.push_back(sys_of);
  GABP_CUDA(cudaMalloc(&misc, sizeof(int) * 2 + sizeof(unsigned int) * 2));
  fr.p.push_back(misc);
  bar = reinterpret_cast<unsigned int *>(misc + 2);
  GABP_CUDA(cudaMemsetAsync(misc, 0, sizeof(int) * 2 + sizeof(unsigned int) * 2, h->stream));
  kg_init<<<nsys, kBlock, 0, h->stream>>>(nsys, st, acc, d_off, sys_of);
  const bool sliced = (shape & kSliced) != 0;
  if (sliced) {
    gabp_status e = ensure_gsell(h, nsys, off_host);
    if (e != GABP_OK) return e;
    const size_t Ea = std::max<size_t>(1, (size_t)h->gsl->Es);
    GABP_CUDA(cudaMemsetAsync(h->gsl->MP[0], 0, sizeof(float) * Ea, h->stream));
    GABP_CUDA(cudaMemsetAsync(h->gsl->MP[1], 0, sizeof(float) * Ea, h->stream));
  }
  kg_rows_init<<<blocks_for(g.n, kBlock, h->max_blocks), kBlock, 0, h->stream>>>(
      g.n, g.rp, g.ad, g.ad32, w.NP[0], sliced ? nullptr : w.MP[0], sliced ? nullptr : w.MP[1], x);
  GABP_CUDA(cudaGetLastError());
  GridArgs a;
  a.n = g.n; a.nsys = nsys; a.sys_of = sys_of;
  a.rp = g.rp; a.ci = g.ci; a.av = g.av32; a.ad = g.ad32;
  a.rowptr = g.rowptr; a.col = g.col; a.val = g.val;
  a.MP0 = w.MP[0]; a.MP1 = w.MP[1]; a.NP0 = w.NP[0]; a.NP1 = w.NP[1]; a.NP2 = w.NP[2];
  a.CF = w.CF; a.invP = w.invP;
  a.H0 = w.H[0]; a.H1 = w.H[1]; a.NH0 = w.NH[0]; a.NH1 = w.NH[1]; a.NH2 = w.NH[2];
  a.rhs = w.rhs32; a.b = b; a.x = x;
  a.ns = 0; a.srow = a.sp = a.ssys = nullptr;
  if (sliced) {  // the slot arrays of the sliced layout
    GSell *L = h->gsl;
    a.ns = L->ns; a.srow = L->srow; a.sp = L->sp; a.ssys = L->ssys;
    a.ci = L->sci; a.av = L->sav;
    a.MP0 = L->MP[0]; a.MP1 = L->MP[1]; a.H0 = L->H[0]; a.H1 = L->H[1]; a.CF = L->CF;
  }
  a.st = st; a.acc = acc; a.bar = bar; a.active = misc; a.err = misc + 1;
  a.tol = tol; a.inner_tol = h->opt.inner_tol; a.prec_thr = std::ldexp(1.0, -h->opt.prec_stop_log2);
  a.inner_max = h->opt.inner_max_iter; a.max_refine = h->opt.max_refine; a.max_iter = max_iter;
  // every system needs at most: precision cap + COEF + (RESID + inner cap + UPDATE) per step + final RESID
  const long long bound = (long long)kGPrecCap + 2 +
                          (long long)h->opt.max_refine * (std::min(h->opt.inner_max_iter, std::max(1, max_iter)) + 2) + 1;
  a.max_rounds = (int)std::min<long long>(bound, 0x7fffffff);
  void (*kern)(GridArgs) = grid_kernel(shape);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int grid = per_sm * h->num_sms;
  {
    // about four chunks per warp or more, so that the round's slowest warp has little more work
    // than the average one; longer chunks (fewer accumulator flushes) when the rows allow
    const int lanes = shape & 0xff;
    const long long warps = (long long)grid * (kBlock / 32);
    const long long steps_per_warp = sliced ? ((long long)a.ns + warps - 1) / warps
                                            : ((long long)g.n * lanes + 32LL * warps - 1) / (32LL * warps);
    a.chunk = (int)std::max(1LL, std::min<long long>(kGChunkMax, steps_per_warp / 4));
  }
  cudaEvent_t e0, e1;
  GABP_CUDA(cudaEventCreate(&e0));
  GABP_CUDA(cudaEventCreate(&e1));
  cudaEventRecord(e0, h->stream);
  void *args[] = {&a};
  cudaError_t le = cudaLaunchCooperativeKernel((void *)kern, dim3(grid), dim3(kBlock), args, 0, h->stream);
  cudaEventRecord(e1, h->stream);
  h->prof.launches += 3;
  if (le == cudaSuccess) le = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (le == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (le != cudaSuccess) return cuda_fail(le, "gabp_solve_systems grid kernel");
  if (ms_out) *ms_out = ms;
  // results: status / rounds / refinement steps / relative residual per system
  std::vector<SysState> S(nsys);
  int err = 0;
  GABP_CUDA(cudaMemcpyAsync(S.data(), st, sizeof(SysState) * nsys, cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaMemcpyAsync(&err, misc + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  std::vector<int> res(3 * nsys);
  std::vector<double> rel(nsys);
  for (int s = 0; s < nsys; ++s) {
    res[s] = err ? (int)GABP_TIMEOUT : S[s].status;
    res[nsys + s] = S[s].Tp + S[s].inner_total;
    res[2 * nsys + s] = S[s].steps;
    rel[s] = S[s].bb > 0.0 ? std::sqrt(S[s].rr / S[s].bb) : 0.0;
  }
  GABP_CUDA(cudaMemcpyAsync(d_status, res.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, h->stream));
  GABP_CUDA(cudaMemcpyAsync(d_iters, res.data() + nsys, sizeof(int) * nsys, cudaMemcpyHostToDevice, h->stream));
  GABP_CUDA(cudaMemcpyAsync(d_refine, res.data() + 2 * nsys, sizeof(int) * nsys, cudaMemcpyHostToDevice, h->stream));
  GABP_CUDA(cudaMemcpyAsync(d_relres, rel.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return GABP_OK;
}

}  // namespace gabp
