// fixloop.cu -- the single-loop form of the convergence fix (Chapter "Fixing
// convergence of GaBP"): instead of solving (A + Gamma) x^(t+1) = b + Gamma x^(t)
// by a full GaBP run per outer step, ONE GaBP round (Algorithm 2, information
// form, parallel schedule) on J' = A + Gamma is run per outer step, and the node
// potentials move by the damped update
//   h^(t+1) = (1 - s) h^(t) + s (b + Gamma x^(t)),     x^(0) = 0, h^(1) = b.
// The messages are never restarted; at the fixed point h = b + Gamma x and
// (A + Gamma) x = h, i.e. A x = b.  FP64 throughout; the stop rule is the
// residual of A x = b (the original matrix).
//
// Round t reads the messages and node records of round t-1 and writes those of
// round t (two stores, as solve64.cu).  A node record holds {P~_k, h~_k} as the
// senders' round t needs them: the message sums of round t-1 plus the potential
// of round t (the record is written after the node's potential update).
#include "gabp_internal.cuh"
#include "devutil.cuh"

#include <algorithm>
#include <cmath>

namespace gabp {

namespace {

struct ArgsSL {
  int n;
  const int *__restrict__ rp;
  const int *__restrict__ ci;
  const int *__restrict__ rev;
  const double *__restrict__ av;
  const double *__restrict__ ad;   // A_ii
  const double *__restrict__ gam;  // Gamma_ii
  const double *__restrict__ b;    // staged right-hand side
  const int *__restrict__ rowptr;
  const int *__restrict__ col;
  const double *__restrict__ val;
  double s;
  double2 *M0, *M1;  // messages {P, h} per slot
  double2 *N0, *N1;  // node records {P~, h~}
  double *hpot;      // node potential h_i of the next round
  double *x;         // x^(t)
  DevCtl *ctl;
  double *partials;
};

__global__ void ksl_init(ArgsSL a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) {
    a.N0[i] = make_double2(a.ad[i] + a.gam[i], a.b[i]);  // no message yet, h^(1) = b
    a.hpot[i] = a.b[i];
    a.x[i] = 0.0;
  }
}

template <int L>
__global__ void __launch_bounds__(kBlock) ksl_round(ArgsSL a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int t = ctl->round + 1;
  const double2 *__restrict__ Min = (t & 1) ? a.M0 : a.M1;
  double2 *__restrict__ Mout = (t & 1) ? a.M1 : a.M0;
  const double2 *__restrict__ Nin = (t & 1) ? a.N0 : a.N1;
  double2 *__restrict__ Nout = (t & 1) ? a.N1 : a.N0;
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  int bad = 0;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int i = base + sw;
    double SP = 0.0, SH = 0.0;
    if (i < a.n)
      for (int e = a.rp[i] + sl; e < a.rp[i + 1]; e += L) {
        const int k = a.ci[e];
        const double A = a.av[e];
        const double2 rv = Min[a.rev[e]];  // message i -> k of round t-1
        const double2 nk = Nin[k];         // k's aggregate with its round-t potential
        const double d = nk.x - rv.x;      // P_{k\i}
        bad |= is_zero64(d);
        const double r = 1.0 / d;
        const double2 m = make_double2(-A * A * r, -A * (nk.y - rv.y) * r);
        Mout[e] = m;
        SP += m.x;
        SH += m.y;
      }
    SP = sub_sum<L>(SP);
    SH = sub_sum<L>(SH);
    if (i < a.n && sl == 0) {
      const double g = a.gam[i], h = a.hpot[i];
      const double P = a.ad[i] + g + SP;
      bad |= is_zero64(P);
      const double xi = (h + SH) / P;
      const double hn = (1.0 - a.s) * h + a.s * (a.b[i] + g * xi);  // the damped potential of round t+1
      a.hpot[i] = hn;
      a.x[i] = xi;
      Nout[i] = make_double2(P, hn + SH);
    }
  }
  if (bad) atomicOr(&ctl->edge_bad, 1);
}

// ||b - A x^(t)||^2 over the full CSR and the decision.
template <int L>
__global__ void __launch_bounds__(kBlock) ksl_decide(ArgsSL a) {
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

__global__ void ksl_bb(int n, const double *__restrict__ b, DevCtl *ctl, double *partials, int max_iter, double tol) {
  double sacc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) sacc = fma(b[i], b[i], sacc);
  double v[1] = {sacc}, tot[1];
  const int modes[1] = {0};
  block_sum<1>(v);
  if (last_block_reduce<1>(v, modes, partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    ctl->round = 0;
    ctl->done = tot[0] == 0.0;
    ctl->status = tot[0] == 0.0 ? GABP_OK : GABP_NOT_CONVERGED;
    ctl->iters = 0;
    ctl->result_round = 0;
    ctl->max_iter = max_iter;
    ctl->bb = tot[0];
    ctl->tol2bb = tol * tol * tot[0];
    ctl->rr = tot[0];
    ctl->edge_bad = 0;
    ctl->no_stop = 0;
    ctl->arrive = 0;
    __threadfence();
  }
}

}  // namespace

void free_wf(gabp_handle h) {
  WorkF &f = h->wf;
  cudaFree(f.M[0]); cudaFree(f.M[1]); cudaFree(f.N[0]); cudaFree(f.N[1]);
  cudaFree(f.hpot); cudaFree(f.bin); cudaFree(f.xin);
  if (h->gSL) cudaGraphExecDestroy(h->gSL);
  h->gSL = nullptr;
  f = WorkF{};
}

// Single-loop convergence fix for one right-hand side; gamma_diag = Gamma (device).
gabp_status solve_fix_single(gabp_handle h, const double *b, double *x, double tol, int max_iter,
                             const double *gamma_diag, int *iters, double *relres) {
  NvtxRange nvtx_("gabp single-loop convergence fix");
  Graph &g = h->g;
  WorkF &f = h->wf;
  const size_t Ea = (size_t)(g.E > 0 ? g.E : 1);
  if (!f.M[0]) {
    GABP_CUDA(cudaMalloc(&f.M[0], sizeof(double2) * Ea));
    GABP_CUDA(cudaMalloc(&f.M[1], sizeof(double2) * Ea));
    GABP_CUDA(cudaMalloc(&f.N[0], sizeof(double2) * g.n));
    GABP_CUDA(cudaMalloc(&f.N[1], sizeof(double2) * g.n));
    GABP_CUDA(cudaMalloc(&f.hpot, sizeof(double) * g.n));
    GABP_CUDA(cudaMalloc(&f.bin, sizeof(double) * g.n));
    GABP_CUDA(cudaMalloc(&f.xin, sizeof(double) * g.n));
  }
  // the captured rounds read and write only handle-owned arrays (Gamma is the handle's; b and x are staged)
  GABP_CUDA(cudaMemcpyAsync(f.bin, b, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, h->stream));
  ArgsSL a;
  a.n = g.n; a.rp = g.rp; a.ci = g.ci; a.rev = g.rev; a.av = g.av; a.ad = g.ad; a.gam = gamma_diag; a.b = f.bin;
  a.rowptr = g.rowptr; a.col = g.col; a.val = g.val; a.s = h->opt.fix_step;
  a.M0 = f.M[0]; a.M1 = f.M[1]; a.N0 = f.N[0]; a.N1 = f.N[1]; a.hpot = f.hpot; a.x = f.xin;
  a.ctl = h->ctl; a.partials = h->partials;
  GABP_CUDA(cudaMemsetAsync(f.M[0], 0, sizeof(double2) * Ea, h->stream));
  ksl_init<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(a);
  ksl_bb<<<blocks_for(g.n, kBlock, h->max_blocks), kBlock, 0, h->stream>>>(g.n, f.bin, h->ctl, h->partials,
                                                                           std::max(1, max_iter), tol);
  GABP_CUDA(cudaGetLastError());
  gabp_status st = read_ctl(h);
  if (st != GABP_OK) return st;
  const double bb = h->ctl_host->bb;
  h->stats.rounds = 0;
  h->stats.edge_updates = -1;
  h->stats.refine_steps = 0;
  if (bb > 0.0) {
    const int L = g.avg_deg >= 12.0 ? 2 : 1;
    // the damping step s is baked into the captured rounds' arguments
    if (h->gSL && h->wf.step != h->opt.fix_step) {
      cudaGraphExecDestroy(h->gSL);
      h->gSL = nullptr;
    }
    h->wf.step = h->opt.fix_step;
    const int key = L;
    gabp_status rs = GABP_OK;
    GABP_DISPATCH_L(L, {
      const int nb = blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, ksl_round<LL>));
      rs = run_rounds(h, &h->gSL, &h->gSL_key, key, [&] {
        ksl_round<LL><<<nb, kBlock, 0, h->stream>>>(a);
        ksl_decide<LL><<<nb, kBlock, 0, h->stream>>>(a);
      }, std::max(1, max_iter), PH_FP64);
    });
    if (rs != GABP_OK) return rs;
  }
  GABP_CUDA(cudaMemcpyAsync(x, f.xin, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  const DevCtl c = *h->ctl_host;
  h->stats.rounds = c.round;
  if (iters) *iters = c.iters;
  if (relres) *relres = bb > 0.0 ? std::sqrt(c.rr / bb) : 0.0;
  return (gabp_status)c.status;
}

}  // namespace gabp
