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
// Layout.  The nodes are relabelled so that every colour class is one
// contiguous range (colour order, index order inside a colour), and every
// row's off-diagonal slots are sorted by the new sender label, so that the
// slots of row j whose sender has colour c form the segment [co[c][j],
// co[c+1][j]).  Pass c updates, in every row outside colour c's range, the
// segment of colour c: exactly the messages sent by the nodes that fire in pass
// c.  Right-hand sides, iterates and marginals are permuted at the boundary.
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
#include "cluster.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>
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

// Slots of new row j (old row oid[j]) in new-sender order: sperm[srp[j] + rank] = e
// (e an off-diagonal slot of the input layout).  A thread ranks its row's slots
// by counting (quadratic in the degree), so rows longer than maxdeg are left to
// the host, which sorts them.
__global__ void ks_sort(int n, const int *__restrict__ srp, const int *__restrict__ oid, const int *__restrict__ rp,
                        const int *__restrict__ ci, const int *__restrict__ nid, int *__restrict__ sperm, int maxdeg) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int i = oid[j], e0 = rp[i], e1 = rp[i + 1], p0 = srp[j];
    if (e1 - e0 > maxdeg) continue;
    for (int e = e0; e < e1; ++e) {
      const int ke = nid[ci[e]];
      int rank = 0;
      for (int f = e0; f < e1; ++f) rank += nid[ci[f]] < ke;
      sperm[p0 + rank] = e;
    }
  }
}

__global__ void ks_gather(int E, const int *__restrict__ sperm, const int *__restrict__ ci, const int *__restrict__ nid,
                          const double *__restrict__ av, int *__restrict__ sci, double *__restrict__ sav,
                          int *__restrict__ inv) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < E) {
    const int e = sperm[p];
    sci[p] = nid[ci[e]];
    sav[p] = av[e];
    inv[e] = p;
  }
}

// Segment bounds co[c * n + j] (c = 0..C) of new row j.
__global__ void ks_offsets(int n, int C, const int *__restrict__ srp, const int *__restrict__ sci,
                           const int *__restrict__ scol, int *__restrict__ co) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int p = srp[j];
    const int p1 = srp[j + 1];
    for (int c = 0; c <= C; ++c) {
      while (p < p1 && scol[sci[p]] < c) ++p;
      co[(size_t)c * n + j] = p;
    }
  }
}

__global__ void ks_refresh(int E, const int *__restrict__ sperm, const double *__restrict__ av,
                           double *__restrict__ sav) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < E) sav[p] = av[sperm[p]];
}

__global__ void ks_rev(int E, const int *__restrict__ sperm, const int *__restrict__ rev, const int *__restrict__ inv,
                       int *__restrict__ srev) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < E) srev[p] = inv[rev[sperm[p]]];
}

// out[j] = in[oid[j]] (old order -> new order), FP64 / FP32
__global__ void ks_perm64(int n, const int *__restrict__ oid, const double *__restrict__ in, double *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = in[oid[j]];
}
__global__ void ks_perm32(int n, const int *__restrict__ oid, const float *__restrict__ in, float *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = in[oid[j]];
}
// out[oid[j]] = in[j] (new order -> old order)
__global__ void ks_unperm64(int n, const int *__restrict__ oid, const double *__restrict__ in, double *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[oid[j]] = in[j];
}

// Row j of the v-th row of a pass that skips the rows [skip0, skip0 + skipn) of
// the colour that fires (they have no segment of their own colour).
__device__ __forceinline__ int pass_row(int v, int skip0, int skipn) { return v < skip0 ? v : v + skipn; }

// ---------------------------------------------------------------------------- FP64 serial sweeps
struct ArgsS64 {
  int n, C;
  const int *__restrict__ co;
  const int *__restrict__ sci;
  const int *__restrict__ srev;
  const int *__restrict__ scol;
  const int *__restrict__ srp;
  const int *__restrict__ oid;
  const double *__restrict__ sav;
  const double *__restrict__ sad;  // A_jj in the new order
  const double *__restrict__ sb;   // b in the new order
  const double *__restrict__ b;    // b in the input order (residual)
  const int *__restrict__ rowptr;
  const int *__restrict__ col;
  const double *__restrict__ val;
  double2 *SM;    // {P, h} per serial slot (message sender -> row)
  double2 *fire;  // {P~, h~} firing aggregate per node (new order)
  double *x;      // iterate in the input order
  double *sPm;    // marginal precisions in the new order
  double *sh1;    // Steffensen (nullptr otherwise): mean messages after a cycle's first sweep
  double *sx0;    // Steffensen: the cycle's starting iterate x_n (input order)
  double *sx1;    // Steffensen: x_{n+1} (input order)
  double *coef;   // precision freeze: coefficient -A_kj / P_k\j per serial slot (freeze != 0)
  int freeze;     // options.freeze_precisions on a plain serial solve
  DevCtl *ctl;
  double *partials;
};

__global__ void ks64_init(ArgsS64 a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < a.n) {
    a.fire[j] = make_double2(a.sad[j], a.sb[j]);  // no message yet: P~ = A_jj, h~ = b_j
    if (a.sx0) a.sx0[a.oid[j]] = a.sb[j] / a.sad[j];  // x^(0)
  }
}

// Loads of data a kernel's own launch writes: from L2 in the cluster kernel (its
// CTAs' L1 caches are not coherent across its barriers), plain otherwise.
template <bool COOP, typename T> __device__ __forceinline__ T ld_mut(const T *p) { return COOP ? __ldcg(p) : *p; }

// Pass c: the nodes of colour c fire (every other row updates its colour-c
// segment), then the rows of colour c + 1 form their firing aggregates.
// With the precision freeze (state fs of the sweep, see freeze_step): a verify
// sweep (fs 1) also compares every new precision message with the one it
// replaces and stores the coefficient -A / P_k\j; a frozen sweep (fs 2) updates
// the mean messages only, with the stored coefficients.  warp / nwarps: this
// warp among the warps that share the pass.
template <int L, bool COOP>
__device__ __forceinline__ void s64_pass_rows(const ArgsS64 &a, int c, int skip0, int skipn, int fs, int warp,
                                              int nwarps, int &bad, int &moving) {
  const int cn = c + 1 == a.C ? 0 : c + 1;
  const int nv = a.n - skipn;
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  for (int base = warp * RPW; base < nv; base += nwarps * RPW) {
    const int v = base + sw;
    const int j = pass_row(v, skip0, skipn);
    double P = 0.0, h = 0.0;
    bool fires_next = false;
    if (v < nv) {
      const int s0 = a.co[(size_t)c * a.n + j], s1 = a.co[(size_t)(c + 1) * a.n + j];
      if (fs == 2) {
        for (int e = s0 + sl; e < s1; e += L) {
          const double2 fk = ld_mut<COOP>(a.fire + a.sci[e]);
          const double rh = ld_mut<COOP>(reinterpret_cast<const double *>(a.SM + a.srev[e]) + 1);
          reinterpret_cast<double *>(a.SM + e)[1] = ld_mut<COOP>(a.coef + e) * (fk.y - rh);  // mean message only
        }
      } else {
        for (int e = s0 + sl; e < s1; e += L) {
          const int k = a.sci[e];
          const double A = a.sav[e];
          const double2 fk = ld_mut<COOP>(a.fire + k);        // k's aggregate when it fires
          const double2 rv = ld_mut<COOP>(a.SM + a.srev[e]);  // message j -> k as k holds it
          const double d = fk.x - rv.x;                       // P_{k\j}
          bad |= is_zero64(d);
          const double r = rcp64(d);
          const double2 m = make_double2(-A * A * r, -A * (fk.y - rv.y) * r);
          if (fs == 1) {
            moving |= ulp_apart(m.x, ld_mut<COOP>(a.SM + e).x);  // the message this one replaces
            a.coef[e] = -A * r;
          }
          a.SM[e] = m;
        }
      }
      fires_next = a.scol[j] == cn;
    }
    __syncwarp();
    if (fires_next) {
      for (int e = a.srp[j] + sl; e < a.srp[j + 1]; e += L) {
        const double2 m = ld_mut<COOP>(a.SM + e);
        P += m.x;
        h += m.y;
      }
    }
    P = sub_sum<L>(P);
    h = sub_sum<L>(h);
    if (fires_next && sl == 0) a.fire[j] = make_double2(a.sad[j] + P, a.sb[j] + h);
  }
}

template <int L>
__global__ void __launch_bounds__(kBlock) ks64_pass(ArgsS64 a, int c, int skip0, int skipn) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int fs = a.freeze ? ctl->fstate : -1;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  int bad = 0, moving = 0;
  s64_pass_rows<L, false>(a, c, skip0, skipn, fs, warp, nwarps, bad, moving);
  if (bad) atomicOr(&ctl->edge_bad, 1);
  if (moving) atomicOr(&ctl->fmove, 1);
}

// After a sweep: x = h~ / P~ and P from every current message (Algorithm 1
// step 4), x written in the input order.
// A screening sweep of the precision freeze (fs 0, from the second sweep on) also
// flags a node whose P moved since the previous sweep.
template <int L, bool COOP>
__device__ __forceinline__ void s64_final_rows(const ArgsS64 &a, bool screen, int warp, int nwarps, int &bad,
                                               int &moving) {
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int j = base + sw;
    double P = 0.0, h = 0.0;
    if (j < a.n)
      for (int e = a.srp[j] + sl; e < a.srp[j + 1]; e += L) {
        const double2 m = ld_mut<COOP>(a.SM + e);
        P += m.x;
        h += m.y;
      }
    P = sub_sum<L>(P);
    h = sub_sum<L>(h);
    if (j < a.n && sl == 0) {
      P += a.sad[j];
      h += a.sb[j];
      bad |= is_zero64(P);
      if (screen) moving |= ulp_apart(P, ld_mut<COOP>(a.sPm + j));
      a.sPm[j] = P;
      a.x[a.oid[j]] = h / P;
    }
  }
}

template <int L>
__global__ void __launch_bounds__(kBlock) ks64_final(ArgsS64 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const bool screen = a.freeze && ctl->fstate == 0 && ctl->round >= 1;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  int bad = 0, moving = 0;
  s64_final_rows<L, false>(a, screen, warp, nwarps, bad, moving);
  if (bad) atomicOr(&ctl->edge_bad, 2);
  if (moving) atomicOr(&ctl->fmove, 1);
}

// This lane's share of ||b - A x||^2 for the sweep's x (input order).
template <int L, bool COOP>
__device__ __forceinline__ double s64_resid_rows(const ArgsS64 &a, int warp, int nwarps) {
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  double rr = 0.0;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int i = base + sw;
    double ax = 0.0;
    if (i < a.n)
      for (int p = a.rowptr[i] + sl; p < a.rowptr[i + 1]; p += L) ax = fma(a.val[p], ld_mut<COOP>(a.x + a.col[p]), ax);
    ax = sub_sum<L>(ax);
    if (i < a.n && sl == 0) {
      const double r = a.b[i] - ax;
      rr = fma(r, r, rr);
    }
  }
  return rr;
}

// ||b - A x||^2 of the sweep's x (input order) and the decision (Algorithm 1
// step 3 with the residual rule): breakdown, divergence, convergence, max_iter.
template <int L>
__global__ void __launch_bounds__(kBlock) ks64_decide(ArgsS64 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  double v[1] = {s64_resid_rows<L, false>(a, warp, nwarps)}, tot[1];
  const int modes[1] = {0};
  block_sum<1>(v);
  if (last_block_reduce<1>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    const int t = ctl->round + 1;
    ctl->round = t;
    ctl->rr = tot[0];
    if (a.freeze) {  // the freeze state after this sweep (the first sweep screens nothing)
      const int fs = ctl->fstate;
      if (fs < 2 && (fs == 1 || t >= 2)) freeze_step(ctl, fs, t, (double)ctl->fmove);
      ctl->fmove = 0;
    }
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

// Every sweep of a small graph in one thread-block cluster (up to 16 CTAs of NW
// warps): the passes, the final x and the residual of each sweep are the kernels'
// above, with a cluster barrier where a launch ended; the residual is summed by
// cluster_sums and every warp takes the decision itself (CTA 0 records it), so all
// CTAs leave after the same sweep.  With the precision freeze CTA 0 also advances
// the freeze state, read by every CTA after one more barrier.  cstart: the colour
// classes' first rows (C + 1 entries).
template <int L, int NW>
__global__ void __launch_bounds__(32 * NW) ks64_cluster(ArgsS64 a, const int *__restrict__ cstart, int max_sweeps) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank(), csize = cl.num_blocks();
  __shared__ ClusterPart part[2][NW];
  DevCtl *ctl = a.ctl;
  const int t0 = ctl->round;  // read by every CTA before the first barrier, written only after it
  const double tol2bb = ctl->tol2bb;
  const int max_iter = ctl->max_iter;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warp = (int)(rank * NW) + wib, nwarps = (int)(csize * NW);
  for (int it = 0; it < max_sweeps; ++it) {
    const int t = t0 + 1 + it;
    const int fs = a.freeze ? __ldcg(&ctl->fstate) : -1;
    int ebad = 0, nbad = 0, moving = 0;
    for (int c = 0; c < a.C; ++c) {
      s64_pass_rows<L, true>(a, c, cstart[c], cstart[c + 1] - cstart[c], fs, warp, nwarps, ebad, moving);
      cl.sync();
    }
    s64_final_rows<L, true>(a, a.freeze && fs == 0 && t - 1 >= 1, warp, nwarps, nbad, moving);
    cl.sync();
    const double rr = s64_resid_rows<L, true>(a, warp, nwarps);
    // flags: bit 0 a zero cavity precision, bit 1 a zero node precision, bit 2 a precision moved
    const ClusterSums tot =
        cluster_sums<NW>(cl, part[t & 1], rr, (ebad ? 1 : 0) | (nbad ? 2 : 0) | (moving ? 4 : 0), lane, wib, nwarps);
    const int st = (tot.flags & 3) ? GABP_BREAKDOWN : !isfinite(tot.rr) ? GABP_DIVERGED
                   : tot.rr <= tol2bb ? GABP_OK : t >= max_iter ? GABP_NOT_CONVERGED : -1;
    if (rank == 0 && threadIdx.x == 0) {
      ctl->round = t;
      ctl->rr = tot.rr;
      if (a.freeze && fs < 2 && (fs == 1 || t >= 2)) freeze_step(ctl, fs, t, (tot.flags & 4) ? 1.0 : 0.0);
      if (st >= 0) {
        ctl->edge_bad = tot.flags & 3;
        ctl->status = st; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
      }
    }
    if (st >= 0) break;
    if (a.freeze) cl.sync();  // the freeze state CTA 0 wrote is read by every CTA next sweep
  }
  cl.sync();  // no CTA leaves while a peer may still read its shared memory
}

// The one-cluster sweeps with the state in the cluster's shared memory (plain
// sweeps, no freeze): CTA r owns the R = NW 32 / L rows from r R on -- their
// messages (the slots of those rows), firing aggregates, marginal precisions and
// iterate -- and every row keeps one group of L lanes for the whole solve.  A slot
// reads the sender's firing aggregate and the reverse message from the sender's
// CTA (the reverse slot lies in the sender's row) through distributed shared
// memory; every write stays in its own CTA.  Messages, aggregates and iterates
// are ks64_pass / ks64_final's, bit for bit; the residual adds each row's terms in
// slot order.  The state is loaded at the start and written back at the end.
struct ChipS {
  int R;  // rows a CTA
  int S;  // slots of the largest CTA
};
__host__ __device__ inline size_t chip_s_bytes(const ChipS &c, int C, bool stf) {
  return (size_t)32 * c.S + (size_t)c.R * (52 + 4 * (size_t)(C + 1)) + (stf ? (size_t)8 * c.S + (size_t)16 * c.R : 0);
}

// STF: Steffensen's iterations (ks64_steff_a / ks64_steff_b's steps, the cycle's scalar step from a
// cluster sum): per slot the mean message after a cycle's first sweep, per row x_n and x_{n+1}.
template <int L, int NW, bool STF>
__global__ void __launch_bounds__(32 * NW) ks64_chip(ArgsS64 a, ChipS c, int max_sweeps) {
  namespace cg = cooperative_groups;
  constexpr int NT = 32 * NW, RPW = 32 / L;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank(), csize = cl.num_blocks();
  const int R = c.R, S = c.S;
  extern __shared__ __align__(16) unsigned char smem[];
  double2 *SMl = reinterpret_cast<double2 *>(smem);  // messages into the own rows, by local slot
  double2 *firel = SMl + S;                          // firing aggregates, by local row
  double *savl = reinterpret_cast<double *>(firel + R);
  double *sPml = savl + S, *sadl = sPml + R, *sbl = sadl + R, *xl = sbl + R;
  double *sh1l = xl + R;                               // STF: mean messages after a cycle's first sweep
  double *x0l = sh1l + (STF ? S : 0), *x1l = x0l + R;  // STF: x_n, x_{n+1}
  int *kref = reinterpret_cast<int *>(STF ? x1l + R : xl + R);  // sender: owner rank << 24 | its local row
  int *rref = kref + S;                         // reverse slot: owner rank << 24 | its local slot
  int *coL = rref + S;                          // [(C + 1) x R] colour segment bounds, local slots
  int *scoll = coL + (size_t)(a.C + 1) * R;
  __shared__ ClusterPart part[2][NW];
  __shared__ ClusterPart2 part2[2][NW];
  DevCtl *ctl = a.ctl;
  const int t0 = ctl->round;
  const double tol2bb = ctl->tol2bb;
  const int max_iter = ctl->max_iter;
  const int j0 = min((int)rank * R, a.n), jn = min(j0 + R, a.n);
  const int e0 = a.srp[j0], eN = a.srp[jn];
  for (int q = threadIdx.x; q < eN - e0; q += NT) {
    const int e = e0 + q, k = a.sci[e], ok = k / R;
    SMl[q] = a.SM[e];
    savl[q] = a.sav[e];
    kref[q] = (ok << 24) | (k - ok * R);
    rref[q] = (ok << 24) | (a.srev[e] - a.srp[ok * R]);
  }
  for (int r = threadIdx.x; r < R; r += NT) {
    const int j = j0 + r;
    if (j < jn) {
      firel[r] = a.fire[j];
      sPml[r] = a.sPm[j];
      sadl[r] = a.sad[j];
      sbl[r] = a.sb[j];
      scoll[r] = a.scol[j];
      for (int cc = 0; cc <= a.C; ++cc) coL[(size_t)cc * R + r] = a.co[(size_t)cc * a.n + j] - e0;
      if (STF) x0l[r] = a.sx0[a.oid[j]];  // x^(0)
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L, wib = threadIdx.x >> 5;
  const int r = wib * RPW + sw;  // this lane group's row, for the whole solve
  const int j = j0 + r;
  const bool has = j < jn;
  const int q0 = has ? a.srp[j] - e0 : 0, q1 = has ? a.srp[j + 1] - e0 : 0;
  const int myc = has ? scoll[r] : -1;
  const int lane_nw = (int)(csize * NW);
  cl.sync();  // every CTA's state is in place before any peer reads it
  int ran = 0;
  for (int it = 0; it < max_sweeps; ++it) {
    const int t = t0 + 1 + it;
    int ebad = 0, nbad = 0;
    for (int cc = 0; cc < a.C; ++cc) {  // pass cc: the nodes of colour cc fire
      const int cn = cc + 1 == a.C ? 0 : cc + 1;
      if (has) {
        const int s0 = coL[(size_t)cc * R + r], s1 = coL[(size_t)(cc + 1) * R + r];
        for (int q = s0 + sl; q < s1; q += L) {
          const double A = savl[q];
          const int kr = kref[q], rf = rref[q];
          const double2 fk = *cl.map_shared_rank(firel + (kr & 0xffffff), (unsigned)(kr >> 24));  // k fires
          const double2 rv = *cl.map_shared_rank(SMl + (rf & 0xffffff), (unsigned)(rf >> 24));  // j -> k
          const double d = fk.x - rv.x;  // P_{k\j}
          ebad |= is_zero64(d);
          const double rc = rcp64(d);
          SMl[q] = make_double2(-A * A * rc, -A * (fk.y - rv.y) * rc);
        }
      }
      __syncwarp();
      const bool fires_next = has && myc == cn;
      double P = 0.0, h = 0.0;
      if (fires_next)
        for (int q = q0 + sl; q < q1; q += L) {
          const double2 m = SMl[q];
          P += m.x;
          h += m.y;
        }
      P = sub_sum<L>(P);
      h = sub_sum<L>(h);
      if (fires_next && sl == 0) firel[r] = make_double2(sadl[r] + P, sbl[r] + h);
      cl.sync();
    }
    {  // x = h~ / P~ and P from every current message
      double P = 0.0, h = 0.0;
      if (has)
        for (int q = q0 + sl; q < q1; q += L) {
          const double2 m = SMl[q];
          P += m.x;
          h += m.y;
        }
      P = sub_sum<L>(P);
      h = sub_sum<L>(h);
      if (has && sl == 0) {
        P += sadl[r];
        h += sbl[r];
        nbad |= is_zero64(P);
        sPml[r] = P;
        xl[r] = h / P;
      }
    }
    if (STF) {
      __syncwarp();
      if (t & 1) {  // a cycle's first sweep: keep its mean messages and iterate
        if (has) {
          for (int q = q0 + sl; q < q1; q += L) sh1l[q] = SMl[q].y;
          if (sl == 0) x1l[r] = xl[r];
        }
      } else {  // after its second: lam = <d, D> / <D, D>, the mean messages and x moved by it
        double sdD = 0.0, sDD = 0.0;
        if (has && sl == 0) {
          const double x0 = x0l[r], x1 = x1l[r], x2 = xl[r];
          const double d = x2 - x1, D = d - (x1 - x0);
          sdD = fma(d, D, sdD);
          sDD = fma(D, D, sDD);
        }
        const double2 tot2 = cluster_sums2<NW>(cl, part2[t & 2 ? 1 : 0], sdD, sDD, lane, wib, lane_nw);
        double lam = tot2.y > 0.0 ? tot2.x / tot2.y : 0.0;
        lam = isfinite(lam) ? lam : 0.0;
        double P = 0.0, h = 0.0;
        if (has)
          for (int q = q0 + sl; q < q1; q += L) {
            const double2 m = SMl[q];
            const double hn = m.y - lam * (m.y - sh1l[q]);
            SMl[q].y = hn;
            P += m.x;
            h += hn;
          }
        P = sub_sum<L>(P);
        h = sub_sum<L>(h);
        if (has && sl == 0) {
          P += sadl[r];
          h += sbl[r];
          const double x = h / P;
          xl[r] = x;
          x0l[r] = x;
          if (myc == 0) firel[r] = make_double2(P, h);
        }
      }
    }
    cl.sync();
    double rr = 0.0;
    {  // ||b - A x||^2, row j: b_j - (A_jj x_j + sum_k A_jk x_k)
      double ax = 0.0;
      if (has)
        for (int q = q0 + sl; q < q1; q += L) {
          const int kr = kref[q];
          ax = fma(savl[q], *cl.map_shared_rank(xl + (kr & 0xffffff), (unsigned)(kr >> 24)), ax);
        }
      ax = sub_sum<L>(ax);
      if (has && sl == 0) {
        const double res = sbl[r] - fma(sadl[r], xl[r], ax);
        rr = res * res;
      }
    }
    ++ran;
    const ClusterSums tot =
        cluster_sums<NW>(cl, part[t & 1], rr, (ebad ? 1 : 0) | (nbad ? 2 : 0), lane, wib, lane_nw);
    const int st = (tot.flags & 3) ? GABP_BREAKDOWN : !isfinite(tot.rr) ? GABP_DIVERGED
                   : tot.rr <= tol2bb ? GABP_OK : t >= max_iter ? GABP_NOT_CONVERGED : -1;
    if (rank == 0 && threadIdx.x == 0) {
      ctl->round = t;
      ctl->rr = tot.rr;
      if (st >= 0) {
        ctl->edge_bad = tot.flags & 3;
        ctl->status = st; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
      }
    }
    if (st >= 0) break;
  }
  // back to the global arrays (the last sweep wrote before its barriers)
  if (ran > 0) {
    for (int q = threadIdx.x; q < eN - e0; q += NT) a.SM[e0 + q] = SMl[q];
    for (int rr2 = threadIdx.x; rr2 < jn - j0; rr2 += NT) {
      const int jj = j0 + rr2;
      a.fire[jj] = firel[rr2];
      a.sPm[jj] = sPml[rr2];
      a.x[a.oid[jj]] = xl[rr2];
    }
  }
  cl.sync();  // no CTA leaves while a peer may still read its shared memory
}

// Steffensen's iterations on the serial schedule (Sec. "Convergence Acceleration"):
// sweeps pair into cycles.  After the first sweep of a cycle (t odd) its mean
// messages and iterate are kept; after the second (t even) the last block forms
// the scalar step lam = <d, D> / <D, D> (d = x_{n+2} - x_{n+1},
// D = x_{n+2} - 2 x_{n+1} + x_n; 0 where nothing moves or the quotient is not finite).
__global__ void __launch_bounds__(kBlock) ks64_steff_a(ArgsS64 a, int E) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int t = ctl->round + 1;  // the sweep just completed
  const int stride = gridDim.x * kBlock, g0 = blockIdx.x * kBlock + threadIdx.x;
  if (t & 1) {
    for (int e = g0; e < E; e += stride) a.sh1[e] = a.SM[e].y;
    for (int i = g0; i < a.n; i += stride) a.sx1[i] = a.x[i];
    return;
  }
  double sdD = 0.0, sDD = 0.0;
  for (int i = g0; i < a.n; i += stride) {
    const double x0 = a.sx0[i], x1 = a.sx1[i], x2 = a.x[i];
    const double d = x2 - x1, D = d - (x1 - x0);
    sdD = fma(d, D, sdD);
    sDD = fma(D, D, sDD);
  }
  double v[2] = {sdD, sDD}, tot[2];
  const int modes[2] = {0, 0};
  block_sum<2>(v);
  if (last_block_reduce<2>(v, modes, a.partials, &ctl->arrive, tot) && threadIdx.x == 0) {
    const double lam = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
    ctl->lam = isfinite(lam) ? lam : 0.0;
    ctl->arrive = 0;
    __threadfence();
  }
}

// After a cycle's second sweep: "y replaces x_n and GaBP runs again".  The mean
// messages move by the cycle's step, h <- h - lam (h - h_{n+1}) (precisions
// stay), and the iterate, the next cycle's x_n and the firing aggregates of the
// colour that fires first are rebuilt from them (x = y exactly when the
// precisions are stationary).
template <int L>
__global__ void __launch_bounds__(kBlock) ks64_steff_b(ArgsS64 a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done || ((ctl->round + 1) & 1)) return;
  const double lam = ctl->lam;
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  for (int base = warp * RPW; base < a.n; base += nwarps * RPW) {
    const int j = base + sw;
    double P = 0.0, h = 0.0;
    if (j < a.n)
      for (int e = a.srp[j] + sl; e < a.srp[j + 1]; e += L) {
        const double2 m = a.SM[e];
        const double hn = m.y - lam * (m.y - a.sh1[e]);
        a.SM[e].y = hn;
        P += m.x;
        h += hn;
      }
    P = sub_sum<L>(P);
    h = sub_sum<L>(h);
    if (j < a.n && sl == 0) {
      P += a.sad[j];
      h += a.sb[j];
      const double x = h / P;
      a.x[a.oid[j]] = x;
      a.sx0[a.oid[j]] = x;
      if (a.scol[j] == 0) a.fire[j] = make_double2(P, h);
    }
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
  c->maxrel = 0.0;
  c->arrive = 0;
  c->edge_bad = 0;
  c->no_stop = 0;
  c->fstate = c->pstat = c->fround = c->pfail = c->fchecks = c->fmove = 0;
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

// serial slot -> input-layout slot (messages read-back)
__global__ void ks_unpermute(int E, const int *__restrict__ sperm, const double2 *__restrict__ SM, double2 *M) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < E) M[sperm[p]] = SM[p];
}

// ---------------------------------------------------------------------------- FP32 serial mean sweeps
struct ArgsS32 {
  int n, C;
  const int *__restrict__ co;
  const int *__restrict__ sci;
  const int *__restrict__ scol;
  const int *__restrict__ srp;
  const float2 *__restrict__ sCF;  // {c_in, c_out} in the serial slot order
  const float *__restrict__ srhs;  // inner right-hand side, new order
  const float *__restrict__ sinvP; // 1 / P~, new order
  float *sH;     // mean message per serial slot
  float *hfire;  // h~_j at j's last firing (new order)
  DevCtl *ctl;
  double *partials;
};

__global__ void ks32_init(int n, const int *__restrict__ oid, const float *__restrict__ rhs, float *__restrict__ srhs,
                          float *__restrict__ hfire) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    const float r = rhs[oid[j]];
    srhs[j] = r;
    hfire[j] = r;  // no message yet: h~_j = r_j
  }
}

// Pass c of a frozen-coefficient mean sweep (L lanes per row, U slots per lane
// with their loads issued together).  The sweep's stop test adds
// ||x^fire_new - x^fire_old||^2 and ||x^fire_new||^2 over the rows forming a new
// firing aggregate in this pass (every row once per sweep) and decides after
// the last pass: estimated error <= itol ||x|| (from the second sweep), a
// non-finite value, or max_iter sweeps.
template <int L, int U>
__global__ void __launch_bounds__(kBlock) ks32_pass(ArgsS32 a, int c, int skip0, int skipn) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int cn = c + 1 == a.C ? 0 : c + 1;
  const int nv = a.n - skipn;
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  float dxx = 0.f, xx = 0.f;
  for (int base = warp * RPW; base < nv; base += nwarps * RPW) {
    const int v = base + sw;
    const int j = pass_row(v, skip0, skipn);
    bool fires_next = false;
    float h = 0.f;  // this lane's share of the new aggregate
    int s0 = 0, s1 = 0;
    if (v < nv) {
      const float hj = a.hfire[j];
      s0 = a.co[(size_t)c * a.n + j];
      s1 = a.co[(size_t)(c + 1) * a.n + j];
      for (int eb = s0 + sl; eb < s1; eb += L * U) {
        int k[U];
        float2 cf[U];
        float hs[U], hk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = eb + u * L;
          if (e < s1) { k[u] = __ldcs(a.sci + e); cf[u] = __ldcs(a.sCF + e); hs[u] = a.sH[e]; }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (eb + u * L < s1) hk[u] = a.hfire[k[u]];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = eb + u * L;
          if (e < s1) {
            const float hout = cf[u].y * (hj - hs[u]);  // message j -> k when j last fired
            const float hn = cf[u].x * (hk[u] - hout);  // message k -> j, k firing now
            a.sH[e] = hn;
            h += hn;
          }
        }
      }
      fires_next = a.scol[j] == cn;
    }
    if (fires_next) {  // the rest of the row (the segment's new messages are in h already)
      for (int e = a.srp[j] + sl; e < s0; e += L) h += a.sH[e];
      for (int e = s1 + sl; e < a.srp[j + 1]; e += L) h += a.sH[e];
    }
    h = sub_sum<L>(h);
    if (fires_next && sl == 0) {
      const float hn = a.srhs[j] + h, ip = a.sinvP[j];
      const float dx = (hn - a.hfire[j]) * ip, xn = hn * ip;
      dxx = fmaf(dx, dx, dxx);
      xx = fmaf(xn, xn, xx);
      a.hfire[j] = hn;
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
      const double dd = ctl->rr, x2 = ctl->xx, prev = ctl->maxrel;
      ctl->maxrel = dd;
      // a serial sweep contracts without the sign alternation of the parallel
      // rounds, so the step underestimates the error: error ~ step q / (1 - q)
      // with q = ||dx_t|| / ||dx_{t-1}||, taken between 1 and 4 steps (a ratio
      // near 1 is FP32 noise at the end of the solve, not slow convergence)
      double f2 = 1.0;
      if (t >= 3 && prev > 0.0) {
        const double q = sqrt(dd / prev);
        f2 = q < 0.8 ? fmax(1.0, (q / (1.0 - q)) * (q / (1.0 - q))) : 16.0;
      }
      if (!isfinite(dd) || !isfinite(x2)) {
        ctl->status = GABP_DIVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
      } else if (t >= 2 && dd * f2 <= ctl->tol2bb * x2) {
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

// x (input order) += d, d_j = h~_j^fire / P~_j
__global__ void ks32_update(int n, const int *__restrict__ oid, const float *__restrict__ hfire,
                            const float *__restrict__ sinvP, double *__restrict__ x) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[oid[j]] += (double)(hfire[j] * sinvP[j]);
}

__global__ void ks32_permute_cf(int E, const int *__restrict__ sperm, const float2 *__restrict__ CF, float2 *sCF) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < E) sCF[p] = CF[sperm[p]];
}

int serial_lanes64(const Graph &g) { return g.avg_deg >= 24.0 ? 4 : (g.avg_deg >= 8.0 ? 2 : 1); }

}  // namespace

void free_ws(gabp_handle h) {
  WorkS &s = h->ws;
  cudaFree(s.colour); cudaFree(s.co); cudaFree(s.sperm); cudaFree(s.sci); cudaFree(s.srev); cudaFree(s.sav);
  cudaFree(s.oid); cudaFree(s.nid); cudaFree(s.srp); cudaFree(s.scol); cudaFree(s.sad); cudaFree(s.sb);
  cudaFree(s.SM); cudaFree(s.fire); cudaFree(s.sPm); cudaFree(s.sCF); cudaFree(s.sH); cudaFree(s.hfire);
  cudaFree(s.srhs); cudaFree(s.sinvP); cudaFree(s.bin); cudaFree(s.xin); cudaFree(s.sh1); cudaFree(s.sx0);
  cudaFree(s.sx1); cudaFree(s.coef); cudaFree(s.dcstart);
  if (h->gS64) cudaGraphExecDestroy(h->gS64);
  if (h->gS32) cudaGraphExecDestroy(h->gS32);
  h->gS64 = h->gS32 = nullptr;
  s = WorkS{};
}

// Colouring, the colour-grouped relabelling and the colour-sorted slot layout
// (once per handle).
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
  // Every pass colours at least the lowest uncoloured node; the number of passes
  // is the longest chain of index-increasing neighbours (about 3 m on an m^3
  // grid, but n on a path numbered along itself).  After kColourPasses device
  // passes the host finishes the greedy colouring in index order, which gives
  // the same colouring: the device passes coloured exactly what the sequential
  // first-fit would have.
  constexpr int kColourPasses = 64;
  int hm[2] = {1, 0};
  for (int done_passes = 0; hm[0] > 0 && done_passes < kColourPasses; done_passes += 8) {
    for (int k = 0; k < 8; ++k) {
      GABP_CUDA(cudaMemsetAsync(misc, 0, sizeof(int), h->stream));
      ks_colour<<<nb, kBlock, 0, h->stream>>>(n, g.rp, g.ci, s.colour, misc, misc + 1);
    }
    GABP_CUDA(cudaMemcpyAsync(hm, misc, sizeof(int) * 2, cudaMemcpyDeviceToHost, h->stream));
    GABP_CUDA(cudaStreamSynchronize(h->stream));
  }
  // relabelling: colour classes contiguous, index order inside (a stable counting sort)
  std::vector<int> col(n), rp(n + 1), oid(n), nid(n), srp(n + 1), scol(n);
  GABP_CUDA(cudaMemcpyAsync(col.data(), s.colour, sizeof(int) * n, cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaMemcpyAsync(rp.data(), g.rp, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  int maxdeg = 0;
  for (int i = 0; i < n; ++i) maxdeg = std::max(maxdeg, rp[i + 1] - rp[i]);
  constexpr int kSortDeviceMaxDeg = 256;  // longer rows are sorted on the host
  std::vector<int> ci_h;
  if (hm[0] > 0 || maxdeg > kSortDeviceMaxDeg) {
    ci_h.resize(Ea);
    if (E > 0) {
      GABP_CUDA(cudaMemcpyAsync(ci_h.data(), g.ci, sizeof(int) * (size_t)E, cudaMemcpyDeviceToHost, h->stream));
      GABP_CUDA(cudaStreamSynchronize(h->stream));
    }
  }
  if (hm[0] > 0) {  // sequential first-fit over the nodes still uncoloured, in index order
    std::vector<int> seen(maxdeg + 2, -1);  // colours are at most the degree
    for (int i = 0; i < n; ++i) {
      if (col[i] >= 0) continue;
      for (int e = rp[i]; e < rp[i + 1]; ++e)
        if (ci_h[e] < i) seen[col[ci_h[e]]] = i;  // lower neighbours are coloured by now
      int c = 0;
      while (seen[c] == i) ++c;
      col[i] = c;
      hm[1] = std::max(hm[1], c);
    }
    GABP_CUDA(cudaMemcpyAsync(s.colour, col.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
  }
  s.C = hm[1] + 1;
  s.cstart.assign(s.C + 1, 0);
  for (int i = 0; i < n; ++i) ++s.cstart[col[i] + 1];
  for (int c = 0; c < s.C; ++c) s.cstart[c + 1] += s.cstart[c];
  std::vector<int> fill(s.cstart.begin(), s.cstart.end() - 1);
  for (int i = 0; i < n; ++i) {
    const int j = fill[col[i]]++;
    oid[j] = i;
    nid[i] = j;
  }
  srp[0] = 0;
  for (int j = 0; j < n; ++j) {
    srp[j + 1] = srp[j] + (rp[oid[j] + 1] - rp[oid[j]]);
    scol[j] = col[oid[j]];
  }
  s.srp_h = srp;
  GABP_CUDA(cudaMalloc(&s.dcstart, sizeof(int) * (s.C + 1)));
  GABP_CUDA(cudaMemcpyAsync(s.dcstart, s.cstart.data(), sizeof(int) * (s.C + 1), cudaMemcpyHostToDevice, h->stream));
  s.clu = -1;
  GABP_CUDA(cudaMalloc(&s.oid, sizeof(int) * n));
  GABP_CUDA(cudaMalloc(&s.nid, sizeof(int) * n));
  GABP_CUDA(cudaMalloc(&s.srp, sizeof(int) * (n + 1)));
  GABP_CUDA(cudaMalloc(&s.scol, sizeof(int) * n));
  GABP_CUDA(cudaMalloc(&s.sad, sizeof(double) * n));
  GABP_CUDA(cudaMemcpyAsync(s.oid, oid.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
  GABP_CUDA(cudaMemcpyAsync(s.nid, nid.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
  GABP_CUDA(cudaMemcpyAsync(s.srp, srp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, h->stream));
  GABP_CUDA(cudaMemcpyAsync(s.scol, scol.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
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
  ks_sort<<<nb, kBlock, 0, h->stream>>>(n, s.srp, s.oid, g.rp, g.ci, s.nid, s.sperm, kSortDeviceMaxDeg);
  if (maxdeg > kSortDeviceMaxDeg) {  // long rows: (new sender label, slot) pairs sorted on the host
    std::vector<std::pair<int, int>> key;
    std::vector<int> perm;
    for (int j = 0; j < n; ++j) {
      const int i = oid[j], e0 = rp[i], e1 = rp[i + 1];
      if (e1 - e0 <= kSortDeviceMaxDeg) continue;
      key.clear();
      for (int e = e0; e < e1; ++e) key.emplace_back(nid[ci_h[e]], e);
      std::sort(key.begin(), key.end());
      perm.resize(key.size());
      for (size_t r = 0; r < key.size(); ++r) perm[r] = key[r].second;
      GABP_CUDA(cudaMemcpyAsync(s.sperm + srp[j], perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice,
                                h->stream));
      GABP_CUDA(cudaStreamSynchronize(h->stream));  // perm is refilled for the next long row
    }
  }
  if (E > 0) {
    const int eb = (E + kBlock - 1) / kBlock;
    ks_gather<<<eb, kBlock, 0, h->stream>>>(E, s.sperm, g.ci, s.nid, g.av, s.sci, s.sav, inv);
    ks_rev<<<eb, kBlock, 0, h->stream>>>(E, s.sperm, g.rev, inv, s.srev);
  }
  ks_offsets<<<nb, kBlock, 0, h->stream>>>(n, s.C, s.srp, s.sci, s.scol, s.co);
  ks_perm64<<<(n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(n, s.oid, g.ad, s.sad);
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  s.ready = true;
  return GABP_OK;
}

// New values on the same pattern (gabp_set_values): the serial-order copies of
// A's values follow; the colouring and the layout depend on the pattern only.
gabp_status serial_refresh_values(gabp_handle h) {
  WorkS &s = h->ws;
  if (!s.ready) return GABP_OK;
  Graph &g = h->g;
  if (g.E > 0)
    ks_refresh<<<(g.E + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.E, s.sperm, g.av, s.sav);
  ks_perm64<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, s.oid, g.ad, s.sad);
  GABP_CUDA(cudaGetLastError());
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
  a.n = g.n; a.C = s.C; a.co = s.co; a.sci = s.sci; a.srev = s.srev; a.scol = s.scol; a.srp = s.srp; a.oid = s.oid;
  a.sav = s.sav; a.sad = s.sad; a.sb = s.sb; a.b = b; a.rowptr = g.rowptr; a.col = g.col; a.val = g.val;
  a.SM = s.SM; a.fire = s.fire; a.x = x; a.sPm = s.sPm;
  const bool stf = h->opt.accel == 2;
  a.sh1 = stf ? s.sh1 : nullptr;
  a.sx0 = stf ? s.sx0 : nullptr;
  a.sx1 = stf ? s.sx1 : nullptr;
  a.freeze = h->opt.freeze_precisions && h->opt.accel == 0 && s.coef != nullptr;
  a.coef = a.freeze ? s.coef : nullptr;
  a.ctl = h->ctl; a.partials = h->partials;
  return a;
}

// The one-cluster sweeps: up to 16 CTAs of NW = 2, 4 or 8 warps, the fewest warps a CTA that
// give every warp one group of 32 / L rows in each pass; graphs needing more than 128 warps
// take the launches.
constexpr int kSerialClusterMax = 16;

template <int L, int NW>
static int serial_cluster_fits(gabp_handle h, int cs) {
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
  if (cs > 8) cudaFuncSetAttribute(ks64_cluster<L, NW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  int nc = 0;
  const bool ok = cudaOccupancyMaxActiveClusters(&nc, (void *)ks64_cluster<L, NW>, &cfg) == cudaSuccess && nc > 0;
  cudaGetLastError();
  return ok ? cs : 0;
}

// The on-chip flavour's shared memory for clusters of cs CTAs of NW warps, when it fits (0 if not).
template <int L, int NW, bool STF>
static int serial_chip_bytes(gabp_handle h, int cs, const ChipS &c) {
  const size_t bytes = chip_s_bytes(c, h->ws.C, STF);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  constexpr int kStaticRoom = 1024;  // the kernel's static shared memory fits below
  if (bytes + kStaticRoom > (size_t)optin) return 0;
  // one limit for the function, shared by every handle: the device's whole opt-in room
  if (cudaFuncSetAttribute(ks64_chip<L, NW, STF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - kStaticRoom) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cs > 8) cudaFuncSetAttribute(ks64_chip<L, NW, STF>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(32 * NW);
  cfg.dynamicSmemBytes = bytes;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nc = 0;
  const bool ok = cudaOccupancyMaxActiveClusters(&nc, (void *)ks64_chip<L, NW, STF>, &cfg) == cudaSuccess && nc > 0;
  cudaGetLastError();
  return ok ? (int)bytes : 0;
}

template <int L, int NW>
static void serial_chip_fit(gabp_handle h, int cs) {
  WorkS &s = h->ws;
  const int R = NW * (32 / L), n = h->g.n;
  int64_t smax = 0;
  for (int r = 0; r < cs; ++r) {
    const int a0 = std::min(r * R, n), a1 = std::min(a0 + R, n);
    smax = std::max<int64_t>(smax, s.srp_h[a1] - s.srp_h[a0]);
  }
  if (smax >= (1 << 24)) return;
  const ChipS c{R, (int)smax};
  s.chip_S = c.S;
  s.chip_bytes = serial_chip_bytes<L, NW, false>(h, cs, c);
  s.chip_bytes_stf = serial_chip_bytes<L, NW, true>(h, cs, c);
}

template <int L>
static void serial_cluster_size(gabp_handle h) {
  WorkS &s = h->ws;
  s.clu = 0;
  s.clu_nw = 0;
  s.chip_bytes = s.chip_bytes_stf = 0;
  s.chip_S = 0;
  int attr = 0;
  cudaDeviceGetAttribute(&attr, cudaDevAttrClusterLaunch, h->device);
  if (!attr) return;
  const int64_t warps = ((int64_t)h->g.n + 32 / L - 1) / (32 / L);
  for (int nw : {2, 4, 8}) {
    const int64_t cs = std::max<int64_t>(1, (warps + nw - 1) / nw);
    if (cs > kSerialClusterMax) continue;
    const int c = nw == 2 ? serial_cluster_fits<L, 2>(h, (int)cs)
                  : nw == 4 ? serial_cluster_fits<L, 4>(h, (int)cs) : serial_cluster_fits<L, 8>(h, (int)cs);
    if (c > 0) {
      s.clu = c;
      s.clu_nw = nw;
      if (nw == 2) serial_chip_fit<L, 2>(h, c);
      else if (nw == 4) serial_chip_fit<L, 4>(h, c);
      else serial_chip_fit<L, 8>(h, c);
    }
    return;
  }
}

template <int L, int NW>
static gabp_status serial_cluster_run(gabp_handle h, const ArgsS64 &a, int max_sweeps) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = h->ws.clu;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(h->ws.clu);
  cfg.blockDim = dim3(32 * NW);
  cfg.stream = h->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // plain sweeps (and Steffensen's) with the state on chip where it fits (the same messages and
  // iterates); the freeze's sweeps read it from global memory
  const bool stf = a.sx0 != nullptr;
  const int chip_bytes = stf ? h->ws.chip_bytes_stf : h->ws.chip_bytes;
  const bool chip = !a.freeze && chip_bytes > 0;
  if (chip) cfg.dynamicSmemBytes = chip_bytes;
  const ChipS cs{NW * (32 / L), h->ws.chip_S};
  prof_begin(h);
  const cudaError_t le =
      chip ? (stf ? cudaLaunchKernelEx(&cfg, ks64_chip<L, NW, true>, a, cs, max_sweeps)
                  : cudaLaunchKernelEx(&cfg, ks64_chip<L, NW, false>, a, cs, max_sweeps))
           : cudaLaunchKernelEx(&cfg, ks64_cluster<L, NW>, a, (const int *)h->ws.dcstart, max_sweeps);
  if (le != cudaSuccess) return cuda_fail(le, "FP64 serial cluster sweeps");
  prof_end(h);
  h->prof.launches += 1;
  gabp_status st = read_ctl(h);
  if (st != GABP_OK) return st;
  prof_collect(h, PH_FP64, h->ctl_host->round);
  if (!h->ctl_host->done) {
    set_last_error("FP64 serial cluster sweeps ended without a decision");
    return GABP_ERR_CUDA;
  }
  return GABP_OK;
}

template <int L>
static gabp_status serial_cluster_dispatch(gabp_handle h, const ArgsS64 &a, int max_sweeps) {
  switch (h->ws.clu_nw) {
    case 2: return serial_cluster_run<L, 2>(h, a, max_sweeps);
    case 4: return serial_cluster_run<L, 4>(h, a, max_sweeps);
    default: return serial_cluster_run<L, 8>(h, a, max_sweeps);
  }
}

// Plain FP64 GaBP under the serial schedule; the answer is the x of the last
// sweep (Algorithm 1 step 4 over every current message).
gabp_status solve64_serial(gabp_handle h, const double *b, double *x, double tol, int max_iter, int *iters,
                           double *relres) {
  NvtxRange nvtx_("gabp fp64 serial schedule");
  gabp_status st = serial_prepare(h);
  if (st != GABP_OK) return st;
  Graph &g = h->g;
  WorkS &s = h->ws;
  const size_t Ea = (size_t)(g.E > 0 ? g.E : 1);
  if (!s.SM) {
    GABP_CUDA(cudaMalloc(&s.SM, sizeof(double2) * Ea));
    GABP_CUDA(cudaMalloc(&s.fire, sizeof(double2) * g.n));
    GABP_CUDA(cudaMalloc(&s.sPm, sizeof(double) * g.n));
    GABP_CUDA(cudaMalloc(&s.sb, sizeof(double) * g.n));
    GABP_CUDA(cudaMalloc(&s.bin, sizeof(double) * g.n));
    GABP_CUDA(cudaMalloc(&s.xin, sizeof(double) * g.n));
  }
  if (h->opt.freeze_precisions && h->opt.accel == 0 && !s.coef)  // the frozen coefficients
    GABP_CUDA(cudaMalloc(&s.coef, sizeof(double) * Ea));
  if (h->opt.accel == 2 && !s.sh1) {  // Steffensen's iterations
    GABP_CUDA(cudaMalloc(&s.sh1, sizeof(double) * Ea));
    GABP_CUDA(cudaMalloc(&s.sx0, sizeof(double) * g.n));
    GABP_CUDA(cudaMalloc(&s.sx1, sizeof(double) * g.n));
  }
  // the captured sweeps read and write only the handle's arrays: b and x are staged
  GABP_CUDA(cudaMemcpyAsync(s.bin, b, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, h->stream));
  ArgsS64 a = args_s64(h, s.bin, s.xin);
  const int n1 = (g.n + kBlock - 1) / kBlock;
  ks_perm64<<<n1, kBlock, 0, h->stream>>>(g.n, s.oid, s.bin, s.sb);
  GABP_CUDA(cudaMemsetAsync(s.SM, 0, sizeof(double2) * Ea, h->stream));
  GABP_CUDA(cudaMemsetAsync(s.xin, 0, sizeof(double) * g.n, h->stream));
  ks64_init<<<n1, kBlock, 0, h->stream>>>(a);
  ks_bb<<<blocks_for(g.n, kBlock, h->max_blocks), kBlock, 0, h->stream>>>(g.n, b, h->ctl, h->partials);
  GABP_CUDA(cudaGetLastError());
  if ((st = read_ctl(h)) != GABP_OK) return st;
  const double bb = h->ctl_host->bb;
  h->stats.rounds = 0;
  h->stats.edge_updates = -1;
  h->stats.refine_steps = 0;
  s.valid = true;
  s.result_round = 0;
  const int L = serial_lanes64(g);
  if (bb == 0.0) {  // x = 0 after zero sweeps; P from the zero messages
    ks64_ctl<<<1, 1, 0, h->stream>>>(h->ctl, 1, 1.0, 0.0);
    GABP_DISPATCH_L(L, (ks64_final<LL><<<blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, ks64_final<LL>)),
                                         kBlock, 0, h->stream>>>(a)));
    GABP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * g.n, h->stream));
    GABP_CUDA(cudaMemsetAsync(s.xin, 0, sizeof(double) * g.n, h->stream));
    GABP_CUDA(cudaStreamSynchronize(h->stream));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return GABP_OK;
  }
  ks64_ctl<<<1, 1, 0, h->stream>>>(h->ctl, std::max(1, max_iter), bb, tol * tol);
  GABP_CUDA(cudaGetLastError());
  const bool stf = h->opt.accel == 2;
  const int key = L | (s.C << 8) | (stf ? 1 << 30 : 0) | (a.freeze ? 1 << 29 : 0);
  gabp_status rs = GABP_OK;
  // small graphs: every sweep in one thread-block cluster (Steffensen's step only with the state
  // on chip)
  bool one_launch = false;
  if (L == 1 || L == 2 || L == 4) {
    if (s.clu < 0) {
      if (L == 1) serial_cluster_size<1>(h);
      else if (L == 2) serial_cluster_size<2>(h);
      else serial_cluster_size<4>(h);
    }
    one_launch = s.clu > 0 && (!stf || s.chip_bytes_stf > 0);
    if (one_launch) {
      const int ms = std::max(1, max_iter);
      rs = L == 1 ? serial_cluster_dispatch<1>(h, a, ms)
           : L == 2 ? serial_cluster_dispatch<2>(h, a, ms) : serial_cluster_dispatch<4>(h, a, ms);
      if (rs != GABP_OK) return rs;
    }
  }
  if (!one_launch) GABP_DISPATCH_L(L, {
    const int nb = blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, ks64_pass<LL>));
    const int ab = blocks_for(std::max(g.n, g.E), kBlock, resident_grid(h->num_sms, ks64_steff_a));
    rs = run_rounds(h, &h->gS64, &h->gS64_key, key, [&] {
      for (int c = 0; c < s.C; ++c)
        ks64_pass<LL><<<nb, kBlock, 0, h->stream>>>(a, c, s.cstart[c], s.cstart[c + 1] - s.cstart[c]);
      ks64_final<LL><<<nb, kBlock, 0, h->stream>>>(a);
      if (stf) {
        ks64_steff_a<<<ab, kBlock, 0, h->stream>>>(a, g.E);
        ks64_steff_b<LL><<<nb, kBlock, 0, h->stream>>>(a);
      }
      ks64_decide<LL><<<nb, kBlock, 0, h->stream>>>(a);
    }, std::max(1, max_iter), PH_FP64);
  });
  if (rs != GABP_OK) return rs;
  GABP_CUDA(cudaMemcpyAsync(x, s.xin, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  const DevCtl c = *h->ctl_host;
  h->stats.rounds = c.round;
  h->stats.freeze_round = a.freeze ? c.fround : 0;
  h->stats.freeze_checks = a.freeze ? c.fchecks : 0;
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
  if (!s.valid || !s.sPm) return GABP_ERR_INVALID;
  ks_unperm64<<<(h->g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(h->g.n, s.oid, s.sPm, Pi);
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return GABP_OK;
}

// ---------------------------------------------------------------------------- FP32 serial inner solve
// Frozen coefficients and 1/P~ in the serial order (after every freeze).
gabp_status serial_freeze32(gabp_handle h, const float2 *CF, const float *invP) {
  gabp_status st = serial_prepare(h);
  if (st != GABP_OK) return st;
  Graph &g = h->g;
  WorkS &s = h->ws;
  const size_t Ea = (size_t)(g.E > 0 ? g.E : 1);
  if (!s.sCF) {
    GABP_CUDA(cudaMalloc(&s.sCF, sizeof(float2) * Ea));
    GABP_CUDA(cudaMalloc(&s.sH, sizeof(float) * Ea));
    GABP_CUDA(cudaMalloc(&s.hfire, sizeof(float) * g.n));
    GABP_CUDA(cudaMalloc(&s.srhs, sizeof(float) * g.n));
    GABP_CUDA(cudaMalloc(&s.sinvP, sizeof(float) * g.n));
  }
  if (g.E > 0) ks32_permute_cf<<<(g.E + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.E, s.sperm, CF, s.sCF);
  ks_perm32<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, s.oid, invP, s.sinvP);
  GABP_CUDA(cudaGetLastError());
  return GABP_OK;
}

// Shape (lanes per row, slots per lane) of the FP32 serial pass from the mean
// length of a colour segment.
static int serial_shape32(const Graph &g, int C) {
  const double seg = C > 1 ? g.avg_deg / (C - 1) : 0.0;
  return seg >= 12.0 ? (4 | (2 << 8)) : seg >= 4.0 ? (2 | (4 << 8)) : (1 | (4 << 8));
}

// One inner solve A d = r with serial frozen-coefficient sweeps until
// ||dx|| <= itol ||x|| or cap sweeps.  *sweeps receives the sweep count.
gabp_status serial_inner32(gabp_handle h, const float *rhs, int cap, double itol, int *sweeps, int *status) {
  Graph &g = h->g;
  WorkS &s = h->ws;
  const size_t Ea = (size_t)(g.E > 0 ? g.E : 1);
  ArgsS32 a;
  a.n = g.n; a.C = s.C; a.co = s.co; a.sci = s.sci; a.scol = s.scol; a.srp = s.srp;
  a.sCF = s.sCF; a.srhs = s.srhs; a.sinvP = s.sinvP; a.sH = s.sH; a.hfire = s.hfire;
  a.ctl = h->ctl; a.partials = h->partials;
  GABP_CUDA(cudaMemsetAsync(s.sH, 0, sizeof(float) * Ea, h->stream));
  ks32_init<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, s.oid, rhs, s.srhs, s.hfire);
  ks64_ctl<<<1, 1, 0, h->stream>>>(h->ctl, cap, 1.0, itol * itol);
  GABP_CUDA(cudaGetLastError());
  const int SH = serial_shape32(g, s.C);
  const int key = SH | (s.C << 16);
  gabp_status rs = GABP_OK;
  auto run = [&](auto Lc, auto Uc) {
    constexpr int LL = decltype(Lc)::value, UU = decltype(Uc)::value;
    const int nb = blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, ks32_pass<LL, UU>));
    rs = run_rounds(h, &h->gS32, &h->gS32_key, key, [&] {
      for (int c = 0; c < s.C; ++c)
        ks32_pass<LL, UU><<<nb, kBlock, 0, h->stream>>>(a, c, s.cstart[c], s.cstart[c + 1] - s.cstart[c]);
    }, cap, PH_MEAN32);
  };
  switch (SH) {
    case 4 | (2 << 8): run(std::integral_constant<int, 4>{}, std::integral_constant<int, 2>{}); break;
    case 2 | (4 << 8): run(std::integral_constant<int, 2>{}, std::integral_constant<int, 4>{}); break;
    default: run(std::integral_constant<int, 1>{}, std::integral_constant<int, 4>{}); break;
  }
  if (rs != GABP_OK) return rs;
  const DevCtl c = *h->ctl_host;
  *sweeps = c.round;
  *status = c.status;
  return GABP_OK;
}

// x (input order) += d of the last serial inner solve
gabp_status serial_update32(gabp_handle h, double *X) {
  WorkS &s = h->ws;
  ks32_update<<<(h->g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(h->g.n, s.oid, s.hfire, s.sinvP, X);
  GABP_CUDA(cudaGetLastError());
  return GABP_OK;
}

}  // namespace gabp
