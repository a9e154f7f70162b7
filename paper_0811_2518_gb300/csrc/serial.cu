// serial.cu -- the serial message schedule (Sec. "The Gaussian BP Algorithm",
// the paragraph on parallel vs serial scheduling): ONE message store, updated in
// place, so a message sent earlier in a sweep is already seen by the nodes that
// fire later in the same sweep.
//
// Order.  A sweep fires the nodes colour by colour (colour 0 first), the
// colouring being the greedy one in index order (each node takes the smallest
// colour not used by a lower-indexed neighbour).  Nodes of one colour share no
// edge, so firing a whole colour at once IS firing its nodes one after the
// other: one kernel pass per colour, the sweep being one sequential order.  The
// colouring is computed on the device with Jones-Plassmann passes whose
// priority is the index, which reproduces the sequential greedy colouring
// exactly.
//
// Layout.  Every row's off-diagonal slots are re-sorted by the sender's colour
// (then index): the slots of row i whose sender has colour c form the segment
// [co[c][i], co[c+1][i]).  Pass c updates, in every row, the segment of colour
// c: these are exactly the messages sent by the nodes that fire in pass c.
//
// Pull form.  The message k -> i sent when k fires is computed by row i's
// thread from k's firing aggregate (one gather) and the reverse message i -> k
// as k holds it.  Row i's thread also forms its own firing aggregate at the end
// of pass colour(i) - 1 (mod the number of colours): after that pass no message
// into i changes before i fires.
//   FP64 (the parity path): the reverse message is gathered from row k.
//   FP32 mean (frozen coefficients): the reverse message is recomputed from
//   what row i holds, h_{i->k} = c_out (h~_i^fire - h_{k->i}), because the slot
//   still holds the message k -> i that i used when it last fired (k has not
//   fired since) -- the same recompute identity as the parallel FP32 rounds.
#include "gabp_internal.cuh"
#include "devutil.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace gabp {

namespace {

// ---------------------------------------------------------------------------- colouring
// One Jones-Plassmann pass: an uncoloured node whose lower-indexed neighbours
// are all coloured takes the smallest colour none of them uses.  Colours are
// written once and read through L2 (never a stale L1 line); a read of
// "uncoloured" racing with the neighbour's write only delays a node to a later
// pass.
__global__ void ks_colour(int n, const int *__restrict__ rp, const int *__restrict__ ci, int *colour, int *left,
                          int *maxc) {
  int mine = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (__ldcg(colour + i) >= 0) continue;
    const int e0 = rp[i], e1 = rp[i + 1];
    bool ready = true;
    for (int e = e0; e < e1 && ready; ++e) {
      const int k = ci[e];
      if (k < i && __ldcg(colour + k) < 0) ready = false;  // through L2: other SMs' colours
    }
    if (!ready) {
      ++mine;
      continue;
    }
    int c = 0;
    for (bool used = true; used;) {
      used = false;
      for (int e = e0; e < e1; ++e) {
        const int k = ci[e];
        if (k < i && __ldcg(colour + k) == c) { used = true; ++c; break; }
      }
    }
    colour[i] = c;
    atomicMax(maxc, c);
  }
  if (mine) atomicAdd(left, mine);
}

// Slots of row i in (sender colour, sender) order: sperm[rp[i] + rank] = e.
__global__ void ks_sort(int n, const int *__restrict__ rp, const int *__restrict__ ci, const int *__restrict__ colour,
                        int *__restrict__ sperm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e0 = rp[i], e1 = rp[i + 1];
    for (int e = e0; e < e1; ++e) {
      const long long ke = ((long long)colour[ci[e]] << 32) | (unsigned)ci[e];
      int rank = 0;
      for (int f = e0; f < e1; ++f) {
        const long long kf = ((long long)colour[ci[f]] << 32) | (unsigned)ci[f];
        rank += kf < ke;
      }
      sperm[e0 + rank] = e;
    }
  }
}

// Segment bounds co[c * n + i] (c = 0..C) and the permuted slot arrays.
__global__ void ks_offsets(int n, int C, const int *__restrict__ rp, const int *__restrict__ ci,
                           const int *__restrict__ colour, const int *__restrict__ sperm, int *__restrict__ co) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int p = rp[i];
    const int e1 = rp[i + 1];
    for (int c = 0; c <= C; ++c) {
      while (p < e1 && colour[ci[sperm[p]]] < c) ++p;
      co[(size_t)c * n + i] = p;
    }
  }
}

__global__ void ks_gather(int E, const int *__restrict__ sperm, const int *__restrict__ ci,
                          const double *__restrict__ av, int *__restrict__ sci, double *__restrict__ sav,
                          int *__restrict__ inv) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < E) {
    const int e = sperm[p];
    sci[p] = ci[e];
    sav[p] = av[e];
    inv[e] = p;
  }
}

__global__ void ks_rev(int E, const int *__restrict__ sperm, const int *__restrict__ rev, const int *__restrict__ inv,
                       int *__restrict__ srev) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < E) srev[p] = inv[rev[sperm[p]]];
}

// ---------------------------------------------------------------------------- FP64 serial sweeps
struct ArgsS64 {
  int n, C;
  const int *__restrict__ co;
  const int *__restrict__ sci;
  const int *__restrict__ srev;
  const int *__restrict__ colour;
  const int *__restrict__ rp;
  const double *__restrict__ sav;
  const double *__restrict__ ad;
  const double *__restrict__ b;
  const int *__restrict__ rowptr;
  const int *__restrict__ col;
  const double *__restrict__ val;
  double2 *SM;    // {P, h} per serial slot (message sender -> row)
  double2 *fire;  // {P~, h~} firing aggregate per node
  double *x, *Pm;
  DevCtl *ctl;
  double *partials;
};

__global__ void ks64_init(ArgsS64 a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) a.fire[i] = make_double2(a.ad[i], a.b[i]);  // no message yet: P~ = A_ii, h~ = b_i
}

// Pass c: the nodes of colour c fire (every row updates its colour-c segment),
// then the rows of colour c + 1 form their firing aggregates.
template <int L>
__global__ void __launch_bounds__(kBlock) ks64_pass(ArgsS64 a, int c) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int cn = c + 1 == a.C ? 0 : c + 1;
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  int bad = 0;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int i = base + sw;
    double P = 0.0, h = 0.0;
    bool fires_next = false;
    if (i < a.n) {
      const int s0 = a.co[(size_t)c * a.n + i], s1 = a.co[(size_t)(c + 1) * a.n + i];
      for (int e = s0 + sl; e < s1; e += L) {
        const int k = a.sci[e];
        const double A = a.sav[e];
        const double2 fk = a.fire[k];         // k's aggregate when it fires
        const double2 rv = a.SM[a.srev[e]];   // message i -> k as k holds it
        const double d = fk.x - rv.x;         // P_{k\i}
        bad |= is_zero64(d);
        const double r = rcp64(d);
        a.SM[e] = make_double2(-A * A * r, -A * (fk.y - rv.y) * r);
      }
      fires_next = a.colour[i] == cn;
    }
    __syncwarp();
    if (fires_next) {
      for (int e = a.rp[i] + sl; e < a.rp[i + 1]; e += L) {
        const double2 m = a.SM[e];
        P += m.x;
        h += m.y;
      }
    }
    P = sub_sum<L>(P);
    h = sub_sum<L>(h);
    if (fires_next && sl == 0) a.fire[i] = make_double2(a.ad[i] + P, a.b[i] + h);
  }
  if (bad) atomicOr(&ctl->edge_bad, 1);
}

// After a sweep: x_i = h~_i / P~_i and P_i from every current message into i.
template <int L>
__global__ void __launch_bounds__(kBlock) ks64_final(ArgsS64 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  int bad = 0;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int i = base + sw;
    double P = 0.0, h = 0.0;
    if (i < a.n)
      for (int e = a.rp[i] + sl; e < a.rp[i + 1]; e += L) {
        const double2 m = a.SM[e];
        P += m.x;
        h += m.y;
      }
    P = sub_sum<L>(P);
    h = sub_sum<L>(h);
    if (i < a.n && sl == 0) {
      P += a.ad[i];
      h += a.b[i];
      bad |= is_zero64(P);
      a.Pm[i] = P;
      a.x[i] = h / P;
    }
  }
  if (bad) atomicOr(&ctl->edge_bad, 2);
}

// ||b - A x||^2 of the sweep's x and the decision (Algorithm 1 step 3 with the
// residual rule): breakdown, divergence, convergence, max_iter.
template <int L>
__global__ void __launch_bounds__(kBlock) ks64_decide(ArgsS64 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  double rr = 0.0;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int i = base + sw;
    double ax = 0.0;
    if (i < a.n)
      for (int p = a.rowptr[i] + sl; p < a.rowptr[i + 1]; p += L) ax = fma(a.val[p], a.x[a.col[p]], ax);
    ax = sub_sum<L>(ax);
    if (i < a.n && sl == 0) {
      const double r = a.b[i] - ax;
      rr = fma(r, r, rr);
    }
  }
  double v[1] = {rr}, tot[1];
  const int modes[1] = {0};
  block_sum<1>(v);
  if (last_block_reduce<1>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    const int t = ctl->round + 1;
    ctl->round = t;
    ctl->rr = tot[0];
    if (ctl->edge_bad) {
      ctl->status = GABP_BREAKDOWN; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (!isfinite(tot[0])) {
      ctl->status = GABP_DIVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (tot[0] <= ctl->tol2bb) {
      ctl->status = GABP_OK; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (t >= ctl->max_iter) {
      ctl->status = GABP_NOT_CONVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    }
    ctl->arrive = 0;
    __threadfence();
  }
}

__global__ void ks64_ctl(DevCtl *c, int max_iter, double bb, double tol2) {
  c->round = 0;
  c->done = 0;
  c->status = GABP_NOT_CONVERGED;
  c->iters = 0;
  c->result_round = 0;
  c->max_iter = max_iter;
  c->bb = bb;
  c->tol2bb = tol2 * bb;
  c->rr = 0.0;
  c->xx = 0.0;
  c->arrive = 0;
  c->edge_bad = 0;
  c->no_stop = 0;
}

// ||b||^2 (FP64, deterministic)
__global__ void ks_bb(int n, const double *__restrict__ b, DevCtl *ctl, double *partials) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s = fma(b[i], b[i], s);
  double v[1] = {s}, tot[1];
  const int modes[1] = {0};
  block_sum<1>(v);
  if (last_block_reduce<1>(v, modes, partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    ctl->bb = tot[0];
    ctl->arrive = 0;
    __threadfence();
  }
}

// serial slot -> input-layout slot (messages read-back, gradient-free marginals)
__global__ void ks_unpermute(int E, const int *__restrict__ sperm, const double2 *__restrict__ SM, double2 *M) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < E) M[sperm[p]] = SM[p];
}

// ---------------------------------------------------------------------------- FP32 serial mean sweeps
struct ArgsS32 {
  int n, C;
  const int *__restrict__ co;
  const int *__restrict__ sci;
  const int *__restrict__ colour;
  const int *__restrict__ rp;
  const float2 *__restrict__ sCF;  // {c_in, c_out} in the serial slot order
  const float *__restrict__ rhs;
  const float *__restrict__ invP;
  float *sH;     // mean message per serial slot
  float *hfire;  // h~_i at i's last firing
  DevCtl *ctl;
  double *partials;
};

__global__ void ks32_init(int n, const float *__restrict__ rhs, float *hfire) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) hfire[i] = rhs[i];  // no message yet: h~_i = r_i
}

// Pass c of a frozen-coefficient mean sweep.  The sweep's stop test adds
// ||x^fire_new - x^fire_old||^2 and ||x^fire_new||^2 over the rows that form a
// new firing aggregate in this pass (every row once per sweep) and decides
// after the last pass: ||dx|| <= itol ||x|| (from the second sweep), a
// non-finite value, or max_iter sweeps.
template <int L>
__global__ void __launch_bounds__(kBlock) ks32_pass(ArgsS32 a, int c) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int cn = c + 1 == a.C ? 0 : c + 1;
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  float dxx = 0.f, xx = 0.f;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int i = base + sw;
    float h = 0.f;
    bool fires_next = false;
    if (i < a.n) {
      const float hi = a.hfire[i];
      const int s0 = a.co[(size_t)c * a.n + i], s1 = a.co[(size_t)(c + 1) * a.n + i];
      for (int e = s0 + sl; e < s1; e += L) {
        const int k = a.sci[e];
        const float2 cf = __ldcs(a.sCF + e);
        const float hout = cf.y * (hi - a.sH[e]);  // message i -> k when i last fired
        a.sH[e] = cf.x * (a.hfire[k] - hout);      // message k -> i, k firing now
      }
      fires_next = a.colour[i] == cn;
    }
    __syncwarp();
    if (fires_next)
      for (int e = a.rp[i] + sl; e < a.rp[i + 1]; e += L) h += a.sH[e];
    h = sub_sum<L>(h);
    if (fires_next && sl == 0) {
      const float hn = a.rhs[i] + h, ip = a.invP[i];
      const float dx = (hn - a.hfire[i]) * ip, xn = hn * ip;
      dxx = fmaf(dx, dx, dxx);
      xx = fmaf(xn, xn, xx);
      a.hfire[i] = hn;
    }
  }
  double v[2] = {(double)dxx, (double)xx}, tot[2];
  const int modes[2] = {0, 0};
  block_sum<2>(v);
  if (last_block_reduce<2>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    ctl->rr += tot[0];
    ctl->xx += tot[1];
    if (c == a.C - 1) {  // the sweep is complete
      const int t = ctl->round + 1;
      ctl->round = t;
      const double dd = ctl->rr, x2 = ctl->xx;
      if (!isfinite(dd) || !isfinite(x2)) {
        ctl->status = GABP_DIVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
      } else if (t >= 2 && dd <= ctl->tol2bb * x2) {
        ctl->status = GABP_OK; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
      } else if (t >= ctl->max_iter) {
        ctl->status = GABP_NOT_CONVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
      }
      ctl->rr = 0.0;
      ctl->xx = 0.0;
    }
    ctl->arrive = 0;
    __threadfence();
  }
}

__global__ void ks32_permute_cf(int E, const int *__restrict__ sperm, const float2 *__restrict__ CF, float2 *sCF) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < E) sCF[p] = CF[sperm[p]];
}

int serial_lanes(const Graph &g) { return g.avg_deg >= 24.0 ? 4 : (g.avg_deg >= 8.0 ? 2 : 1); }

}  // namespace

void free_ws(gabp_handle h) {
  WorkS &s = h->ws;
  cudaFree(s.colour); cudaFree(s.co); cudaFree(s.sperm); cudaFree(s.sci); cudaFree(s.srev); cudaFree(s.sav);
  cudaFree(s.SM); cudaFree(s.fire); cudaFree(s.sCF); cudaFree(s.sH); cudaFree(s.hfire);
  if (h->gS64) cudaGraphExecDestroy(h->gS64);
  if (h->gS32) cudaGraphExecDestroy(h->gS32);
  h->gS64 = h->gS32 = nullptr;
  s = WorkS{};
}

// Colouring and the colour-sorted layout (once per handle).
gabp_status serial_prepare(gabp_handle h) {
  WorkS &s = h->ws;
  if (s.ready) return GABP_OK;
  Graph &g = h->g;
  const int n = g.n, E = g.E;
  const size_t Ea = (size_t)(E > 0 ? E : 1);
  GABP_CUDA(cudaMalloc(&s.colour, sizeof(int) * n));
  int *misc = nullptr;  // [0] nodes left, [1] max colour
  GABP_CUDA(cudaMalloc(&misc, sizeof(int) * 2));
  struct F {
    int *p;
    ~F() { cudaFree(p); }
  } fr{misc};
  GABP_CUDA(cudaMemsetAsync(s.colour, 0xff, sizeof(int) * n, h->stream));
  GABP_CUDA(cudaMemsetAsync(misc, 0, sizeof(int) * 2, h->stream));
  const int nb = blocks_for(n, kBlock, h->max_blocks);
  // every pass colours at least the lowest uncoloured node, so n passes always suffice
  int hm[2] = {1, 0};
  for (long long done_passes = 0; hm[0] > 0; ) {
    if (done_passes > n) {
      set_last_error("serial colouring did not finish");
      return GABP_ERR_CUDA;
    }
    for (int k = 0; k < 8; ++k) {
      GABP_CUDA(cudaMemsetAsync(misc, 0, sizeof(int), h->stream));
      ks_colour<<<nb, kBlock, 0, h->stream>>>(n, g.rp, g.ci, s.colour, misc, misc + 1);
    }
    done_passes += 8;
    GABP_CUDA(cudaMemcpyAsync(hm, misc, sizeof(int) * 2, cudaMemcpyDeviceToHost, h->stream));
    GABP_CUDA(cudaStreamSynchronize(h->stream));
  }
  s.C = hm[1] + 1;
  GABP_CUDA(cudaMalloc(&s.co, sizeof(int) * (size_t)(s.C + 1) * n));
  GABP_CUDA(cudaMalloc(&s.sperm, sizeof(int) * Ea));
  GABP_CUDA(cudaMalloc(&s.sci, sizeof(int) * Ea));
  GABP_CUDA(cudaMalloc(&s.srev, sizeof(int) * Ea));
  GABP_CUDA(cudaMalloc(&s.sav, sizeof(double) * Ea));
  int *inv = nullptr;
  GABP_CUDA(cudaMalloc(&inv, sizeof(int) * Ea));
  struct F2 {
    int *p;
    ~F2() { cudaFree(p); }
  } fr2{inv};
  ks_sort<<<nb, kBlock, 0, h->stream>>>(n, g.rp, g.ci, s.colour, s.sperm);
  ks_offsets<<<nb, kBlock, 0, h->stream>>>(n, s.C, g.rp, g.ci, s.colour, s.sperm, s.co);
  if (E > 0) {
    const int eb = (E + kBlock - 1) / kBlock;
    ks_gather<<<eb, kBlock, 0, h->stream>>>(E, s.sperm, g.ci, g.av, s.sci, s.sav, inv);
    ks_rev<<<eb, kBlock, 0, h->stream>>>(E, s.sperm, g.rev, inv, s.srev);
  }
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  s.ready = true;
  return GABP_OK;
}

gabp_status serial_colours(gabp_handle h, int *colour_dev, int *ncolours) {
  gabp_status st = serial_prepare(h);
  if (st != GABP_OK) return st;
  if (colour_dev) GABP_CUDA(cudaMemcpyAsync(colour_dev, h->ws.colour, sizeof(int) * h->g.n,
                                            cudaMemcpyDeviceToDevice, h->stream));
  if (ncolours) *ncolours = h->ws.C;
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return GABP_OK;
}

static ArgsS64 args_s64(gabp_handle h, const double *b, double *x) {
  Graph &g = h->g;
  WorkS &s = h->ws;
  ArgsS64 a;
  a.n = g.n; a.C = s.C; a.co = s.co; a.sci = s.sci; a.srev = s.srev; a.colour = s.colour; a.rp = g.rp;
  a.sav = s.sav; a.ad = g.ad; a.b = b; a.rowptr = g.rowptr; a.col = g.col; a.val = g.val;
  a.SM = s.SM; a.fire = s.fire; a.x = x; a.Pm = s.Pm;
  a.ctl = h->ctl; a.partials = h->partials;
  return a;
}

// Plain FP64 GaBP under the serial schedule; the answer is the x of the last
// sweep (Algorithm 1 step 4 over every current message).
gabp_status solve64_serial(gabp_handle h, const double *b, double *x, double tol, int max_iter, int *iters,
                           double *relres) {
  gabp_status st = serial_prepare(h);
  if (st != GABP_OK) return st;
  Graph &g = h->g;
  WorkS &s = h->ws;
  const size_t Ea = (size_t)(g.E > 0 ? g.E : 1);
  if (!s.SM) {
    GABP_CUDA(cudaMalloc(&s.SM, sizeof(double2) * Ea));
    GABP_CUDA(cudaMalloc(&s.fire, sizeof(double2) * g.n));
    GABP_CUDA(cudaMalloc(&s.Pm, sizeof(double) * g.n));
  }
  ArgsS64 a = args_s64(h, b, x);
  GABP_CUDA(cudaMemsetAsync(s.SM, 0, sizeof(double2) * Ea, h->stream));
  GABP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * g.n, h->stream));
  ks64_init<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(a);
  ks_bb<<<blocks_for(g.n, kBlock, h->max_blocks), kBlock, 0, h->stream>>>(g.n, b, h->ctl, h->partials);
  GABP_CUDA(cudaGetLastError());
  if ((st = read_ctl(h)) != GABP_OK) return st;
  const double bb = h->ctl_host->bb;
  h->stats.rounds = 0;
  h->stats.edge_updates = -1;
  h->stats.refine_steps = 0;
  s.valid = true;
  s.result_round = 0;
  if (bb == 0.0) {  // x = 0 after zero sweeps; P from the zero messages
    ks64_ctl<<<1, 1, 0, h->stream>>>(h->ctl, 1, 1.0, 0.0);
    const int L = serial_lanes(g);
    GABP_DISPATCH_L(L, (ks64_final<LL><<<blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, ks64_final<LL>)),
                                         kBlock, 0, h->stream>>>(a)));
    GABP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * g.n, h->stream));
    GABP_CUDA(cudaStreamSynchronize(h->stream));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return GABP_OK;
  }
  ks64_ctl<<<1, 1, 0, h->stream>>>(h->ctl, std::max(1, max_iter), bb, tol * tol);
  GABP_CUDA(cudaGetLastError());
  const int L = serial_lanes(g);
  const int key = L | (s.C << 8);
  gabp_status rs = GABP_OK;
  GABP_DISPATCH_L(L, {
    const int nb = blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, ks64_pass<LL>));
    rs = run_rounds(h, &h->gS64, &h->gS64_key, key, [&] {
      for (int c = 0; c < s.C; ++c) ks64_pass<LL><<<nb, kBlock, 0, h->stream>>>(a, c);
      ks64_final<LL><<<nb, kBlock, 0, h->stream>>>(a);
      ks64_decide<LL><<<nb, kBlock, 0, h->stream>>>(a);
    }, std::max(1, max_iter), PH_FP64);
  });
  if (rs != GABP_OK) return rs;
  const DevCtl c = *h->ctl_host;
  h->stats.rounds = c.round;
  s.result_round = c.round;
  if (iters) *iters = c.iters;
  if (relres) *relres = std::sqrt(c.rr / bb);
  return (gabp_status)c.status;
}

gabp_status serial_messages64(gabp_handle h, double2 *M_input_layout) {
  WorkS &s = h->ws;
  if (!s.valid || !s.SM) return GABP_ERR_INVALID;
  if (h->g.E > 0)
    ks_unpermute<<<(h->g.E + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(h->g.E, s.sperm, s.SM, M_input_layout);
  GABP_CUDA(cudaGetLastError());
  return GABP_OK;
}

gabp_status serial_marginals64(gabp_handle h, double *Pi) {
  WorkS &s = h->ws;
  if (!s.valid || !s.Pm) return GABP_ERR_INVALID;
  GABP_CUDA(cudaMemcpyAsync(Pi, s.Pm, sizeof(double) * h->g.n, cudaMemcpyDeviceToDevice, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return GABP_OK;
}

// ---------------------------------------------------------------------------- FP32 serial inner solve
// Frozen coefficients in the serial slot order (after every freeze).
gabp_status serial_freeze32(gabp_handle h, const float2 *CF) {
  gabp_status st = serial_prepare(h);
  if (st != GABP_OK) return st;
  Graph &g = h->g;
  WorkS &s = h->ws;
  const size_t Ea = (size_t)(g.E > 0 ? g.E : 1);
  if (!s.sCF) {
    GABP_CUDA(cudaMalloc(&s.sCF, sizeof(float2) * Ea));
    GABP_CUDA(cudaMalloc(&s.sH, sizeof(float) * Ea));
    GABP_CUDA(cudaMalloc(&s.hfire, sizeof(float) * g.n));
  }
  if (g.E > 0) ks32_permute_cf<<<(g.E + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.E, s.sperm, CF, s.sCF);
  GABP_CUDA(cudaGetLastError());
  return GABP_OK;
}

// One inner solve A d = r (rhs32) with serial frozen-coefficient sweeps until
// ||dx|| <= itol ||x|| or cap sweeps; d_i = h~_i^fire / P~_i is left in hfire
// (times invP).  *sweeps receives the sweep count.
gabp_status serial_inner32(gabp_handle h, const float *rhs, const float *invP, int cap, double itol, int *sweeps,
                           int *status) {
  Graph &g = h->g;
  WorkS &s = h->ws;
  const size_t Ea = (size_t)(g.E > 0 ? g.E : 1);
  ArgsS32 a;
  a.n = g.n; a.C = s.C; a.co = s.co; a.sci = s.sci; a.colour = s.colour; a.rp = g.rp;
  a.sCF = s.sCF; a.rhs = rhs; a.invP = invP; a.sH = s.sH; a.hfire = s.hfire;
  a.ctl = h->ctl; a.partials = h->partials;
  GABP_CUDA(cudaMemsetAsync(s.sH, 0, sizeof(float) * Ea, h->stream));
  ks32_init<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, rhs, s.hfire);
  ks64_ctl<<<1, 1, 0, h->stream>>>(h->ctl, cap, 1.0, itol * itol);
  GABP_CUDA(cudaGetLastError());
  const int L = serial_lanes(g);
  const int key = L | (s.C << 8);
  gabp_status rs = GABP_OK;
  GABP_DISPATCH_L(L, {
    const int nb = blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, ks32_pass<LL>));
    rs = run_rounds(h, &h->gS32, &h->gS32_key, key, [&] {
      for (int c = 0; c < s.C; ++c) ks32_pass<LL><<<nb, kBlock, 0, h->stream>>>(a, c);
    }, cap, PH_MEAN32);
  });
  if (rs != GABP_OK) return rs;
  const DevCtl c = *h->ctl_host;
  *sweeps = c.round;
  *status = c.status;
  return GABP_OK;
}

}  // namespace gabp
