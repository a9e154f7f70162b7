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
// ||x||^2, the outer ||r||^2) are gathered per system; after a grid barrier one
// thread per system takes that system's decision (stationary precisions, inner
// tolerance reached -- with the adaptive target of solve32.cu -- outer
// tolerance reached, breakdown, divergence, caps), then a second barrier opens
// the next round.  Systems therefore converge independently, as if solved one
// by one, while each round streams the rows of all running systems at once.
//
// The grid barrier spins on a generation counter with a clock-bounded wait:
// all blocks are co-resident (cooperative launch), so it always completes; if
// it ever did not within ~2 s, the kernel records GABP_TIMEOUT and returns.
#include "gabp_internal.cuh"
#include "devutil.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace gabp {

namespace {

enum : int { PH_PREC = 0, PH_COEF = 1, PH_RESID = 2, PH_INNER = 3, PH_UPDATE = 4, PH_DONE = 5 };
constexpr int kGU = 4;                       // slots per thread whose loads are issued together
constexpr int kGPrecCap = 300;               // precision-round cap per system
constexpr long long kBarrierLimit = 4000000000LL;  // clock cycles (~2 s) before a barrier gives up

struct SysState {
  int phase, t, stable, Tp, Tm, steps, inner_total, status;
  double bb, rr, itol, pad;
};

struct GridArgs {
  int n, nsys;
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

// Bounded grid barrier (all blocks co-resident).  Returns false if it gave up.
__device__ bool grid_barrier(unsigned int *bar, int *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = bar + 1;
    const unsigned int g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (*(volatile int *)err || clock64() - t0 > kBarrierLimit) { ok = 0; break; }
        __nanosleep(64);
      }
    }
    if (!ok) atomicExch(err, 1);
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Accumulate a row's contribution into its system's sums (slot 0: sum; slot 1:
// sum, or max when max1).  When the whole warp works for one system the warp
// reduces first and lane 0 issues the atomics; otherwise each lane does.  A NaN
// in a max survives (it must not read as "stationary").
__device__ __forceinline__ void accumulate(double *acc, int s, double v0, double v1, bool max1, bool has) {
  __syncwarp();
  const int key = has ? s : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  if (peers == 0xffffffffu) {
    if (key < 0) return;
    double a0 = v0, a1 = v1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      const double b1 = __shfl_xor_sync(0xffffffffu, a1, o);
      a1 = max1 ? ((a1 > b1 || a1 != a1) ? a1 : b1) : a1 + b1;
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(acc + 4 * key, a0);
      if (max1)
        atomicMax(reinterpret_cast<unsigned long long *>(acc + 4 * key + 1), (unsigned long long)__double_as_longlong(a1));
      else
        atomicAdd(acc + 4 * key + 1, a1);
    }
  } else if (has) {
    atomicAdd(acc + 4 * s, v0);
    if (max1)
      atomicMax(reinterpret_cast<unsigned long long *>(acc + 4 * s + 1), (unsigned long long)__double_as_longlong(v1));
    else
      atomicAdd(acc + 4 * s + 1, v1);
  }
}

// A system's state as last written by its decision thread (possibly on another
// SM): read through L2.
__device__ __forceinline__ SysState load_state(const SysState *p) {
  SysState S;
  const int4 *q = reinterpret_cast<const int4 *>(p);
  int4 *d = reinterpret_cast<int4 *>(&S);
#pragma unroll
  for (int j = 0; j < (int)(sizeof(SysState) / sizeof(int4)); ++j) d[j] = __ldcg(q + j);
  return S;
}

__global__ void __launch_bounds__(kBlock) kg_solve(GridArgs a) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31, wid = tid >> 5, nw = nth >> 5;
  for (int round = 0; round < a.max_rounds; ++round) {
    // ---------------------------------------------------------------- work pass
    // warp-uniform loop: every lane of a warp runs every iteration (row i = base + lane)
    for (int base = wid * 32; base < a.n; base += nw * 32) {
      const int i = base + lane;
      double c0 = 0.0, c1 = 0.0;
      bool has = false, mx = false;
      int s = -1;
      if (i < a.n) {
      s = a.sys_of[i];
      const SysState S = load_state(a.st + s);
      if (S.phase == PH_PREC) {
        const int t = S.t;
        float *Mc = (t & 1) ? a.MP1 : a.MP0;
        const float *Mo = (t & 1) ? a.MP0 : a.MP1;
        const float *Pm1 = ring(a.NP0, a.NP1, a.NP2, t + 2);
        const float *Pm2 = ring(a.NP0, a.NP1, a.NP2, t + 1);
        float *Pt = ring(a.NP0, a.NP1, a.NP2, t);
        const float Pi2 = t >= 2 ? Pm2[i] : 0.f;
        float acc = 0.f, rel = 0.f;
        int bad = 0;
        const int e1 = a.rp[i + 1];
        for (int eb = a.rp[i]; eb < e1; eb += kGU) {
          int k[kGU];
          float A[kGU], Ps[kGU], Pp[kGU], Pk[kGU];
#pragma unroll
          for (int u = 0; u < kGU; ++u)
            if (eb + u < e1) { k[u] = a.ci[eb + u]; A[u] = a.av[eb + u]; Ps[u] = Mc[eb + u]; Pp[u] = Mo[eb + u]; }
#pragma unroll
          for (int u = 0; u < kGU; ++u)
            if (eb + u < e1) Pk[u] = __ldcg(Pm1 + k[u]);
#pragma unroll
          for (int u = 0; u < kGU; ++u) {
            if (eb + u < e1) {
              const float A2 = A[u] * A[u];
              float Pout = 0.f;
              if (t >= 2) {
                const float d1 = Pi2 - Ps[u];
                bad |= (d1 == 0.f);
                Pout = -A2 / d1;
              }
              const float d2 = Pk[u] - Pout;
              bad |= (d2 == 0.f);
              const float Pn = -A2 / d2;
              Mc[eb + u] = Pn;
              acc += Pn;
              rel = fmaxf(rel, fabsf(Pn - Pp[u]) / fabsf(Pn));
            }
          }
        }
        const float P = a.ad[i] + acc;
        bad |= (P == 0.f);
        Pt[i] = P;
        c0 = (double)bad;
        c1 = (double)rel;
        has = true;
        mx = true;
      } else if (S.phase == PH_COEF) {
        const int T = S.Tp;
        const float *Ms = (T & 1) ? a.MP1 : a.MP0;
        const float *PT = ring(a.NP0, a.NP1, a.NP2, T);
        const float Pi = PT[i];
        for (int e = a.rp[i]; e < a.rp[i + 1]; ++e) {
          const float A = a.av[e];
          const float cout = -A / (Pi - Ms[e]);
          const float cin = -A / (__ldcg(PT + a.ci[e]) - cout * A);
          a.CF[e] = make_float2(cin, cout);
        }
        a.invP[i] = 1.f / Pi;
        a.x[i] = 0.0;
      } else if (S.phase == PH_RESID) {
        double ax = 0.0;
        for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) ax = fma(a.val[p], __ldcg(a.x + a.col[p]), ax);
        const double r = a.b[i] - ax;
        a.rhs[i] = (float)r;
        a.NH0[i] = (float)r;
        for (int e = a.rp[i]; e < a.rp[i + 1]; ++e) a.H0[e] = 0.f;
        c0 = r * r;
        has = true;
      } else if (S.phase == PH_INNER) {
        const int t = S.t;
        float *Hc = (t & 1) ? a.H1 : a.H0;
        const float *Hm1 = ring(a.NH0, a.NH1, a.NH2, t + 2);
        const float *Hm2 = ring(a.NH0, a.NH1, a.NH2, t + 1);
        float *Ht = ring(a.NH0, a.NH1, a.NH2, t);
        const float hi2 = t >= 2 ? Hm2[i] : 0.f;
        float acc = 0.f;
        const int e1 = a.rp[i + 1];
        for (int eb = a.rp[i]; eb < e1; eb += kGU) {
          int k[kGU];
          float2 cf[kGU];
          float hs[kGU], hk[kGU];
#pragma unroll
          for (int u = 0; u < kGU; ++u)
            if (eb + u < e1) { k[u] = a.ci[eb + u]; cf[u] = a.CF[eb + u]; hs[u] = Hc[eb + u]; }
#pragma unroll
          for (int u = 0; u < kGU; ++u)
            if (eb + u < e1) hk[u] = __ldcg(Hm1 + k[u]);
#pragma unroll
          for (int u = 0; u < kGU; ++u) {
            if (eb + u < e1) {
              const float hout = t >= 2 ? cf[u].y * (hi2 - hs[u]) : 0.f;
              const float hn = cf[u].x * (hk[u] - hout);
              Hc[eb + u] = hn;
              acc += hn;
            }
          }
        }
        const float hnew = a.rhs[i] + acc;
        Ht[i] = hnew;
        const float ip = a.invP[i];
        const float xi = hnew * ip, dx = (hnew - Hm1[i]) * ip;
        c0 = (double)(dx * dx);
        c1 = (double)(xi * xi);
        has = true;
      } else if (S.phase == PH_UPDATE) {
        const float *hT = ring(a.NH0, a.NH1, a.NH2, S.Tm);
        a.x[i] += (double)(hT[i] * a.invP[i]);
      }
      }
      accumulate(a.acc, s, c0, c1, mx, has);
    }
    if (!grid_barrier(a.bar, a.err)) return;
    // ---------------------------------------------------------------- decisions, one thread per system
    for (int s = tid; s < a.nsys; s += nth) {
      SysState S = load_state(a.st + s);
      double *ac = a.acc + 4 * s;
      const double v0 = __ldcg(ac), v1 = __ldcg(ac + 1);
      ac[0] = 0.0;
      ac[1] = 0.0;
      switch (S.phase) {
        case PH_PREC: {
          S.stable = (v1 <= a.prec_thr) ? S.stable + 1 : 0;  // a NaN is not stationary
          if (v0 > 0.0) { S.status = GABP_BREAKDOWN; S.phase = PH_DONE; S.Tp = S.t; }
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
        default: break;
      }
      a.st[s] = S;
      if (S.phase != PH_DONE) atomicAdd(a.active, 1);
    }
    if (!grid_barrier(a.bar, a.err)) return;
    const int act = *(volatile int *)a.active;
    if (!grid_barrier(a.bar, a.err)) return;  // everyone has read the count before it is reset
    if (tid == 0) *a.active = 0;
    if (act == 0) return;
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
    for (int e = rp[i]; e < rp[i + 1]; ++e) { MP0[e] = 0.f; MP1[e] = 0.f; }
  }
}

}  // namespace

gabp_status solve_systems_grid(gabp_handle h, int nsys, const int *d_off, const double *b, double *x, double tol,
                               int max_iter, int *d_status, int *d_iters, int *d_refine, double *d_relres,
                               float *ms_out) {
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
  kg_rows_init<<<blocks_for(g.n, kBlock, h->max_blocks), kBlock, 0, h->stream>>>(g.n, g.rp, g.ad, g.ad32, w.NP[0],
                                                                                  w.MP[0], w.MP[1], x);
  GABP_CUDA(cudaGetLastError());
  GridArgs a;
  a.n = g.n; a.nsys = nsys; a.sys_of = sys_of;
  a.rp = g.rp; a.ci = g.ci; a.av = g.av32; a.ad = g.ad32;
  a.rowptr = g.rowptr; a.col = g.col; a.val = g.val;
  a.MP0 = w.MP[0]; a.MP1 = w.MP[1]; a.NP0 = w.NP[0]; a.NP1 = w.NP[1]; a.NP2 = w.NP[2];
  a.CF = w.CF; a.invP = w.invP;
  a.H0 = w.H[0]; a.H1 = w.H[1]; a.NH0 = w.NH[0]; a.NH1 = w.NH[1]; a.NH2 = w.NH[2];
  a.rhs = w.rhs32; a.b = b; a.x = x;
  a.st = st; a.acc = acc; a.bar = bar; a.active = misc; a.err = misc + 1;
  a.tol = tol; a.inner_tol = h->opt.inner_tol; a.prec_thr = std::ldexp(1.0, -h->opt.prec_stop_log2);
  a.inner_max = h->opt.inner_max_iter; a.max_refine = h->opt.max_refine; a.max_iter = max_iter;
  // every system needs at most: precision cap + COEF + (RESID + inner cap + UPDATE) per step + final RESID
  const long long bound = (long long)kGPrecCap + 2 +
                          (long long)h->opt.max_refine * (std::min(h->opt.inner_max_iter, std::max(1, max_iter)) + 2) + 1;
  a.max_rounds = (int)std::min<long long>(bound, 0x7fffffff);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kg_solve, kBlock, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int grid = per_sm * h->num_sms;
  cudaEvent_t e0, e1;
  GABP_CUDA(cudaEventCreate(&e0));
  GABP_CUDA(cudaEventCreate(&e1));
  cudaEventRecord(e0, h->stream);
  void *args[] = {&a};
  cudaError_t le = cudaLaunchCooperativeKernel((void *)kg_solve, dim3(grid), dim3(kBlock), args, 0, h->stream);
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
