// multi.cu -- many independent systems (a block-diagonal A) solved by ONE
// persistent launch: FP32 precision phase, frozen coefficients, FP32 mean
// rounds and FP64 iterative refinement of every system run inside the kernel.
//
// Each system is solved by a team: either a whole thread-block cluster (kCS
// CTAs, for large systems: the rows are split between the CTAs, rounds are
// separated by the hardware cluster barrier, sums travel through distributed
// shared memory) or a single CTA (small systems: __syncthreads only).  No team
// ever waits on another team, so the kernel holds no spin-wait.  A host-side
// scheduler (longest-processing-time first on a cost model of rows + slots)
// assigns large systems to clusters and small ones to CTAs; the size that
// separates them is picked by timing candidates on first use (autotuning).
//
// The arithmetic is that of solve32.cu (recompute form of Algorithm 2 in FP32,
// FP64 residual and update), per system, with each system's own stop rules:
// precision phase to a 2^-20 stationary point, inner solves to
// ||dx|| <= inner_tol ||x||, outer loop to ||b_s - A_s x_s|| <= tol ||b_s||.
#include "gabp_internal.cuh"
#include "devutil.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace cg = cooperative_groups;

namespace gabp {

namespace {

constexpr int kCS = 8;         // CTAs per cluster (portable maximum)
constexpr int kMU = 2;         // slots per thread whose loads are issued together
constexpr int kPrecCap = 300;  // precision-phase round cap per system

struct MultiArgs {
  const int *__restrict__ offsets;  // [nsys + 1] row offsets of the systems
  const int *__restrict__ rp;       // off-diagonal receiver-layout CSR (block diagonal)
  const int *__restrict__ ci;
  const float *__restrict__ av;     // A_ik (FP32)
  const float *__restrict__ ad;     // A_ii (FP32)
  const int *__restrict__ rowptr;   // full FP64 CSR for the residual
  const int *__restrict__ col;
  const double *__restrict__ val;
  float *MP0, *MP1, *NP0, *NP1, *NP2;
  float2 *CF;
  float *invP;
  float *H0, *H1, *NH0, *NH1, *NH2;
  float *rhs;
  const double *b;
  double *x;
  const int *cl_jobs, *cl_start, *cl_count;    // per cluster: systems solved by the whole cluster
  const int *cta_jobs, *cta_start, *cta_count; // per CTA: systems solved by that CTA alone
  int *sys_status, *sys_iters, *sys_refine;
  double *sys_relres;
  double tol, inner_tol;
  int inner_max, max_refine, max_iter;
};

struct Team {
  bool cluster;
  int rank, size;
};

__device__ __forceinline__ float *ring(float *a, float *b, float *c, int t) {
  const int m = t % 3;
  return m == 0 ? a : (m == 1 ? b : c);
}

__device__ __forceinline__ void team_sync(const Team &T) {
  if (T.cluster) {
    __threadfence();
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

// Sum (mode 0) or max (mode 1) of NV per-thread doubles over the team; every
// thread of every CTA of the team receives the same totals (fixed order).
template <int NV, int NT>
__device__ void team_reduce(const Team &T, double (&v)[NV], const int (&mode)[NV], double (&out)[NV]) {
  __shared__ double part[NV];
  double s[NV], m[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) { s[j] = mode[j] ? 0.0 : v[j]; m[j] = mode[j] ? v[j] : -1.0; }
  block_sum_nt<NV, NT>(s);
  block_max_nt<NV, NT>(m);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) part[j] = mode[j] ? m[j] : s[j];
  }
  if (!T.cluster) {
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) out[j] = part[j];
    __syncthreads();
    return;
  }
  cg::cluster_group cl = cg::this_cluster();
  __threadfence();
  cl.sync();
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double acc = mode[j] ? -1.0 : 0.0;
    for (int r = 0; r < T.size; ++r) {
      const double p = *cl.map_shared_rank(&part[j], r);
      acc = mode[j] ? nan_max(acc, p) : acc + p;
    }
    out[j] = acc;
  }
  cl.sync();  // every CTA has read the partials before they are overwritten
}

// One system, solved by team T.  Thread t of rank r handles rows lo + t, lo + t + NT, ...
template <int NT>
__device__ void solve_system(const MultiArgs &a, int s, const Team &T) {
  const int r0 = a.offsets[s], r1 = a.offsets[s + 1];
  const int nrow = r1 - r0;
  const int chunk = (nrow + T.size - 1) / T.size;
  const int lo = min(r1, r0 + T.rank * chunk), hi = min(r1, lo + chunk);
  const int tid = threadIdx.x, nt = blockDim.x;
  int status = GABP_OK, inner_total = 0, steps = 0;
  double relres = 0.0;

  // ---- precision phase (FP32), round 0: zero messages, P~ = A_ii
  for (int i = lo + tid; i < hi; i += nt) {
    a.NP0[i] = a.ad[i];
    for (int e = a.rp[i]; e < a.rp[i + 1]; ++e) { a.MP0[e] = 0.f; a.MP1[e] = 0.f; }
  }
  team_sync(T);
  int stable = 0, Tp = 0;
  for (int t = 1; t <= kPrecCap; ++t) {
    float *Mc = (t & 1) ? a.MP1 : a.MP0;
    const float *Mo = (t & 1) ? a.MP0 : a.MP1;
    const float *Pm1 = ring(a.NP0, a.NP1, a.NP2, t + 2);
    const float *Pm2 = ring(a.NP0, a.NP1, a.NP2, t + 1);
    float *Pt = ring(a.NP0, a.NP1, a.NP2, t);
    float rel = 0.f;
    int bad = 0;
    for (int i = lo + tid; i < hi; i += nt) {
      const float Pi2 = t >= 2 ? Pm2[i] : 0.f;
      float acc = 0.f;
      const int e1 = a.rp[i + 1];
      for (int eb = a.rp[i]; eb < e1; eb += kMU) {
        int k[kMU];
        float A[kMU], Ps[kMU], Pp[kMU], Pk[kMU];
#pragma unroll
        for (int u = 0; u < kMU; ++u)
          if (eb + u < e1) { k[u] = a.ci[eb + u]; A[u] = a.av[eb + u]; Ps[u] = Mc[eb + u]; Pp[u] = Mo[eb + u]; }
#pragma unroll
        for (int u = 0; u < kMU; ++u)
          if (eb + u < e1) Pk[u] = __ldcg(Pm1 + k[u]);
#pragma unroll
        for (int u = 0; u < kMU; ++u) {
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
            rel = nan_max(rel, rel_change(Pn, Pp[u]));
          }
        }
      }
      const float P = a.ad[i] + acc;
      bad |= (P == 0.f);
      Pt[i] = P;
    }
    double v[2] = {(double)bad, (double)rel}, o[2];
    const int md[2] = {0, 1};
    team_reduce<2, NT>(T, v, md, o);  // also orders this round's writes before the next round's reads
    Tp = t;
    if (o[0] > 0.0) { status = GABP_BREAKDOWN; break; }
    stable = (o[1] <= 9.5367431640625e-7) ? stable + 1 : 0;  // a NaN is not stationary
    if (stable >= 2) break;
  }
  if (status == GABP_OK) {
    // ---- freeze coefficients and 1/P~
    const float *Ms = (Tp & 1) ? a.MP1 : a.MP0;
    const float *PT = ring(a.NP0, a.NP1, a.NP2, Tp);
    for (int i = lo + tid; i < hi; i += nt) {
      const float Pi = PT[i];
      for (int e = a.rp[i]; e < a.rp[i + 1]; ++e) {
        const float A = a.av[e];
        const float cout = -A / (Pi - Ms[e]);
        const float cin = -A / (__ldcg(PT + a.ci[e]) - cout * A);
        a.CF[e] = make_float2(cin, cout);
      }
      a.invP[i] = 1.f / Pi;
      a.x[i] = 0.0;
    }
    team_sync(T);
    // ---- refinement loop
    double bb = 0.0, rr = 0.0;
    for (int it = 0;; ++it) {
      // residual r = b - A x (FP64) over my rows; FP32 copy seeds the inner solve
      double acc_rr = 0.0;
      for (int i = lo + tid; i < hi; i += nt) {
        double ax = 0.0;
        for (int p = a.rowptr[i]; p < a.rowptr[i + 1]; ++p) ax = fma(a.val[p], __ldcg(a.x + a.col[p]), ax);
        const double r = a.b[i] - ax;
        acc_rr = fma(r, r, acc_rr);
        a.rhs[i] = (float)r;
        a.NH0[i] = (float)r;
        for (int e = a.rp[i]; e < a.rp[i + 1]; ++e) a.H0[e] = 0.f;
      }
      double v[1] = {acc_rr}, o[1];
      const int md[1] = {0};
      team_reduce<1, NT>(T, v, md, o);
      rr = o[0];
      if (it == 0) bb = rr;
      if (bb == 0.0 || rr <= a.tol * a.tol * bb) { status = GABP_OK; break; }
      if (!isfinite(rr)) { status = GABP_DIVERGED; break; }
      if (steps >= a.max_refine || inner_total >= a.max_iter) { status = GABP_NOT_CONVERGED; break; }
      // inner FP32 mean iteration from zero messages, to the reduction still needed
      int Tm = 0;
      const int cap = min(a.inner_max, max(1, a.max_iter - inner_total));
      const double need = 0.1 * a.tol * sqrt(bb / rr);
      const double itol = fmin(a.inner_tol, fmax(1e-6, need));
      bool div = false;
      for (int t = 1; t <= cap; ++t) {
        float *Hc = (t & 1) ? a.H1 : a.H0;
        const float *Hm1 = ring(a.NH0, a.NH1, a.NH2, t + 2);
        const float *Hm2 = ring(a.NH0, a.NH1, a.NH2, t + 1);
        float *Ht = ring(a.NH0, a.NH1, a.NH2, t);
        float dxx = 0.f, xx = 0.f;
        for (int i = lo + tid; i < hi; i += nt) {
          const float hi2 = t >= 2 ? Hm2[i] : 0.f;
          float acc = 0.f;
          const int e1 = a.rp[i + 1];
          for (int eb = a.rp[i]; eb < e1; eb += kMU) {
            int k[kMU];
            float2 cf[kMU];
            float hs[kMU], hk[kMU];
#pragma unroll
            for (int u = 0; u < kMU; ++u)
              if (eb + u < e1) { k[u] = a.ci[eb + u]; cf[u] = a.CF[eb + u]; hs[u] = Hc[eb + u]; }
#pragma unroll
            for (int u = 0; u < kMU; ++u)
              if (eb + u < e1) hk[u] = __ldcg(Hm1 + k[u]);
#pragma unroll
            for (int u = 0; u < kMU; ++u) {
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
          dxx = fmaf(dx, dx, dxx);
          xx = fmaf(xi, xi, xx);
        }
        double v2[2] = {(double)dxx, (double)xx}, o2[2];
        const int md2[2] = {0, 0};
        team_reduce<2, NT>(T, v2, md2, o2);
        Tm = t;
        if (!isfinite(o2[0]) || !isfinite(o2[1])) { div = true; break; }
        if (t >= 2 && o2[0] <= itol * itol * o2[1]) break;
      }
      inner_total += Tm;
      if (div) { status = GABP_DIVERGED; break; }
      const float *hT = ring(a.NH0, a.NH1, a.NH2, Tm);
      for (int i = lo + tid; i < hi; i += nt) a.x[i] += (double)(hT[i] * a.invP[i]);
      ++steps;
      team_sync(T);
    }
    relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  } else {
    for (int i = lo + tid; i < hi; i += nt) a.x[i] = 0.0;
  }
  if (T.rank == 0 && tid == 0) {
    a.sys_status[s] = status;
    a.sys_iters[s] = inner_total + Tp;
    a.sys_relres[s] = relres;
    a.sys_refine[s] = steps;
  }
  team_sync(T);
}

// Register cap: 64 per thread (65536 / (NT * blocks)), so at least 1024 threads
// per SM are resident -- the kernel is latency bound and needs warps in flight.
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) km_solve(MultiArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  const int cid = blockIdx.x / kCS;
  // 1) systems solved by the whole cluster, together
  Team tc{true, crank, kCS};
  for (int q = 0; q < a.cl_count[cid]; ++q) solve_system<NT>(a, a.cl_jobs[a.cl_start[cid] + q], tc);
  // 2) systems solved by this CTA alone
  Team ts{false, 0, 1};
  for (int q = 0; q < a.cta_count[blockIdx.x]; ++q)
    solve_system<NT>(a, a.cta_jobs[a.cta_start[blockIdx.x] + q], ts);
}

__global__ void km_diag32(int n, const double *__restrict__ ad, float *__restrict__ d32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d32[i] = (float)ad[i];
}

// Systems must not couple: every column of a system's rows lies inside the system.
__global__ void km_check(int nsys, const int *__restrict__ offsets, const int *__restrict__ rowptr,
                         const int *__restrict__ col, int *flag) {
  const int s = blockIdx.x;
  if (s >= nsys) return;
  const int r0 = offsets[s], r1 = offsets[s + 1];
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x)
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
      if (col[p] < r0 || col[p] >= r1) atomicOr(flag, 1);
}

}  // namespace

struct MultiSched {
  int nclusters = 0;
  std::vector<int> cl_jobs, cl_start, cl_count, cta_jobs, cta_start, cta_count;
};

// Longest-processing-time-first assignment on the cost model rows + slots.
static MultiSched schedule(const std::vector<int> &rows, const std::vector<int> &slots, int nclusters,
                           long long big_threshold) {
  const int nsys = (int)rows.size(), ncta = nclusters * kCS;
  std::vector<int> order(nsys);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> cost(nsys);
  for (int s = 0; s < nsys; ++s) cost[s] = (double)rows[s] + (double)slots[s];
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<double> load(ncta, 0.0);
  std::vector<std::vector<int>> clj(nclusters), ctj(ncta);
  for (int s : order) {
    if ((long long)rows[s] + slots[s] >= big_threshold) {
      int best = 0;
      double bl = 1e300;
      for (int c = 0; c < nclusters; ++c) {
        double m = 0.0;
        for (int j = 0; j < kCS; ++j) m = std::max(m, load[c * kCS + j]);
        if (m < bl) { bl = m; best = c; }
      }
      clj[best].push_back(s);
      for (int j = 0; j < kCS; ++j) load[best * kCS + j] = bl + cost[s] / kCS;
    } else {
      const int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      ctj[best].push_back(s);
      load[best] += cost[s];
    }
  }
  MultiSched S;
  S.nclusters = nclusters;
  for (int c = 0; c < nclusters; ++c) {
    S.cl_start.push_back((int)S.cl_jobs.size());
    S.cl_count.push_back((int)clj[c].size());
    S.cl_jobs.insert(S.cl_jobs.end(), clj[c].begin(), clj[c].end());
  }
  for (int g = 0; g < ncta; ++g) {
    S.cta_start.push_back((int)S.cta_jobs.size());
    S.cta_count.push_back((int)ctj[g].size());
    S.cta_jobs.insert(S.cta_jobs.end(), ctj[g].begin(), ctj[g].end());
  }
  if (S.cl_jobs.empty()) S.cl_jobs.push_back(0);
  if (S.cta_jobs.empty()) S.cta_jobs.push_back(0);
  return S;
}

static gabp_status collect_systems(gabp_handle h, int nsys, const std::vector<int> &slots, const int *d_res,
                                   const double *d_rel, float ms, int *status_host, int *iters_host,
                                   double *relres_host);

gabp_status solve_systems(gabp_handle h, int nsys, const int *offsets_host, const double *b, double *x, double tol,
                          int max_iter, int *status_host, int *iters_host, double *relres_host) {
  NvtxRange nvtx_("gabp independent systems");
  Graph &g = h->g;
  if (nsys < 1 || !offsets_host || offsets_host[0] != 0 || offsets_host[nsys] != g.n) return GABP_ERR_INVALID;
  for (int s = 0; s < nsys; ++s)
    if (offsets_host[s + 1] <= offsets_host[s]) return GABP_ERR_INVALID;
  gabp_status st = ensure_w32(h, 1);
  if (st != GABP_OK) return st;
  Work32 &w = h->w32;
  // per-system sizes from the host copy of the off-diagonal row pointer
  std::vector<int> rp_h(g.n + 1);
  GABP_CUDA(cudaMemcpyAsync(rp_h.data(), g.rp, sizeof(int) * (g.n + 1), cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  std::vector<int> rows(nsys), slots(nsys);
  for (int s = 0; s < nsys; ++s) {
    rows[s] = offsets_host[s + 1] - offsets_host[s];
    slots[s] = rp_h[offsets_host[s + 1]] - rp_h[offsets_host[s]];
  }
  struct Free {
    std::vector<void *> p;
    ~Free() { for (void *q : p) cudaFree(q); }
  } fr;
  int *d_off = nullptr, *d_flag = nullptr, *d_res = nullptr, *d_sched = nullptr;
  double *d_rel = nullptr;
  GABP_CUDA(cudaMalloc(&d_off, sizeof(int) * (nsys + 1)));
  fr.p.push_back(d_off);
  GABP_CUDA(cudaMalloc(&d_flag, sizeof(int)));
  fr.p.push_back(d_flag);
  GABP_CUDA(cudaMalloc(&d_res, sizeof(int) * 3 * nsys));
  fr.p.push_back(d_res);
  GABP_CUDA(cudaMalloc(&d_rel, sizeof(double) * nsys));
  fr.p.push_back(d_rel);
  GABP_CUDA(cudaMemcpyAsync(d_off, offsets_host, sizeof(int) * (nsys + 1), cudaMemcpyHostToDevice, h->stream));
  GABP_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), h->stream));
  km_check<<<nsys, kBlock, 0, h->stream>>>(nsys, d_off, g.rowptr, g.col, d_flag);
  int flag = 0;
  GABP_CUDA(cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  if (flag) {
    set_last_error("gabp_solve_systems: an edge couples two systems");
    return GABP_ERR_INVALID;
  }
  km_diag32<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, g.ad, g.ad32);
  GABP_CUDA(cudaGetLastError());

  // launch configuration of one wave of clusters for a block size NT
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  auto config = [&](int NT, int *nclusters) {
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = h->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(kCS);
    int nc = 0;
    cudaError_t e = NT == 1024 ? cudaOccupancyMaxActiveClusters(&nc, km_solve<1024>, &cfg)
                  : NT == 512  ? cudaOccupancyMaxActiveClusters(&nc, km_solve<512>, &cfg)
                               : cudaOccupancyMaxActiveClusters(&nc, km_solve<256>, &cfg);
    if (e != cudaSuccess || nc < 1) {
      cudaGetLastError();
      nc = std::max(1, h->num_sms / kCS);
    }
    cfg.gridDim = dim3(nc * kCS);
    *nclusters = nc;
    return cfg;
  };

  MultiArgs a;
  a.offsets = d_off;
  a.rp = g.rp; a.ci = g.ci; a.av = g.av32; a.ad = g.ad32;
  a.rowptr = g.rowptr; a.col = g.col; a.val = g.val;
  a.MP0 = w.MP[0]; a.MP1 = w.MP[1]; a.NP0 = w.NP[0]; a.NP1 = w.NP[1]; a.NP2 = w.NP[2];
  a.CF = w.CF; a.invP = w.invP;
  a.H0 = w.H[0]; a.H1 = w.H[1]; a.NH0 = w.NH[0]; a.NH1 = w.NH[1]; a.NH2 = w.NH[2];
  a.rhs = w.rhs32; a.b = b; a.x = x;
  a.sys_status = d_res; a.sys_iters = d_res + nsys; a.sys_refine = d_res + 2 * nsys; a.sys_relres = d_rel;
  a.tol = tol; a.inner_tol = h->opt.inner_tol; a.inner_max = h->opt.inner_max_iter;
  a.max_refine = h->opt.max_refine; a.max_iter = max_iter;

  // one run of the persistent kernel with a given block size and cluster / single-CTA split
  auto run = [&](int NT, long long big, float *ms) -> gabp_status {
    int nclusters = 1;
    cudaLaunchConfig_t cfg = config(NT, &nclusters);
    MultiSched S = schedule(rows, slots, nclusters, big);
    std::vector<int> packed;
    auto put = [&](const std::vector<int> &v) {
      size_t at = packed.size();
      packed.insert(packed.end(), v.begin(), v.end());
      return at;
    };
    const size_t o1 = put(S.cl_jobs), o2 = put(S.cl_start), o3 = put(S.cl_count), o4 = put(S.cta_jobs),
                 o5 = put(S.cta_start), o6 = put(S.cta_count);
    if (d_sched) cudaFree(d_sched);
    d_sched = nullptr;
    GABP_CUDA(cudaMalloc(&d_sched, sizeof(int) * packed.size()));
    GABP_CUDA(cudaMemcpyAsync(d_sched, packed.data(), sizeof(int) * packed.size(), cudaMemcpyHostToDevice, h->stream));
    a.cl_jobs = d_sched + o1; a.cl_start = d_sched + o2; a.cl_count = d_sched + o3;
    a.cta_jobs = d_sched + o4; a.cta_start = d_sched + o5; a.cta_count = d_sched + o6;
    cudaEvent_t e0, e1;
    GABP_CUDA(cudaEventCreate(&e0));
    GABP_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, h->stream);
    cudaError_t le = NT == 1024 ? cudaLaunchKernelEx(&cfg, km_solve<1024>, a)
                   : NT == 512  ? cudaLaunchKernelEx(&cfg, km_solve<512>, a)
                                : cudaLaunchKernelEx(&cfg, km_solve<256>, a);
    cudaEventRecord(e1, h->stream);
    h->prof.launches += 1;
    if (le == cudaSuccess) le = cudaEventSynchronize(e1);
    float t = 0.f;
    if (le == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (le != cudaSuccess) return cuda_fail(le, "gabp_solve_systems kernel");
    *ms = t;
    return GABP_OK;
  };
  struct SchedFree {
    int **p;
    ~SchedFree() { if (*p) cudaFree(*p); }
  } sf{&d_sched};
  float ms = 0.f;
  auto finish = [&](float t) -> gabp_status {
    return collect_systems(h, nsys, slots, d_res, d_rel, t, status_host, iters_host, relres_host);
  };
  auto run_grid_shape = [&](int shape, float *t) {
    return solve_systems_grid(h, nsys, d_off, offsets_host, b, x, tol, max_iter, d_res, d_res + nsys, d_res + 2 * nsys,
                              d_rel, shape, t);
  };
  // grid-kernel shape: the lanes option, else the tuned one, else tune it now
  // (each candidate one complete run; the fastest is kept)
  const int mode = h->opt.multi_split > 0 ? 2 : h->opt.multi_mode ? h->opt.multi_mode : h->multi_mode;
  auto run_grid = [&](float *t) -> gabp_status {
    int shape = 0;
    if (h->opt.lanes >= 1 && h->opt.lanes <= 8) shape = h->opt.lanes | ((h->opt.lanes >= 4 ? 2 : 4) << 8);
    else if (mode != 3 || (h->multi_grid_shape & kSliced)) shape = h->multi_grid_shape;
    if (shape) return run_grid_shape(shape, t);
    // one run of every candidate, then a second run of the two fastest: the one with the smaller
    // total of its two runs is kept (a single run can be off by a few percent)
    float t1 = 1e30f, t2 = 1e30f;
    int s1 = 0, s2 = 0;
    for (int c : kGridShapes) {
      if (mode == 3 && !(c & kSliced)) continue;  // the sliced layout's shapes only
      float tc = 0.f;
      gabp_status e = run_grid_shape(c, &tc);
      if (e != GABP_OK) return e;
      if (tc < t1) { t2 = t1; s2 = s1; t1 = tc; s1 = c; }
      else if (tc < t2) { t2 = tc; s2 = c; }
    }
    shape = s1;
    if (s2) {
      float r1 = 0.f, r2 = 0.f;
      gabp_status e = run_grid_shape(s1, &r1);
      if (e == GABP_OK) e = run_grid_shape(s2, &r2);
      if (e != GABP_OK) return e;
      if (t2 + r2 < t1 + r1) shape = s2;
    }
    h->multi_grid_shape = shape;
    return run_grid_shape(shape, t);
  };
  // kernel choice: the options may force the grid-persistent kernel (mode 1) or
  // teams (mode 2, or any fixed split); otherwise the first call on a handle
  // times both and later calls reuse the faster one
  if (mode == 1 || mode == 3) {
    if ((st = run_grid(&ms)) != GABP_OK) return st;
    return finish(ms);
  }
  int NT = h->multi_nt ? h->multi_nt : 512;
  if (h->opt.multi_split > 0 || (mode == 2 && h->multi_big)) {
    if ((st = run(NT, h->opt.multi_split > 0 ? h->opt.multi_split : h->multi_big, &ms)) != GABP_OK) return st;
    return finish(ms);
  }
  float grid_ms = 1e30f;
  if (mode == 0 && (st = run_grid(&grid_ms)) != GABP_OK) return st;
  // autotune block size, then the size above which a system gets a whole
  // cluster: each candidate is one complete run; the fastest is kept
  float best = 1e30f;
  const int nts[3] = {256, 512, 1024};
  for (int c : nts) {
    if ((st = run(c, 20000, &ms)) != GABP_OK) return st;
    if (ms < best) { best = ms; NT = c; }
  }
  const long long cands[3] = {1LL << 40, 60000, 6000};
  long long split = 20000;
  for (long long c : cands) {
    if ((st = run(NT, c, &ms)) != GABP_OK) return st;
    if (ms < best) { best = ms; split = c; }
  }
  h->multi_big = split;
  h->multi_nt = NT;
  if (best <= grid_ms) {
    if (mode == 0) h->multi_mode = 2;
    if ((st = run(NT, split, &ms)) != GABP_OK) return st;
  } else {
    h->multi_mode = 1;
    if ((st = run_grid(&ms)) != GABP_OK) return st;
  }
  return finish(ms);
}

// per-system results of the last multi-system run (device arrays) back to the caller
static gabp_status collect_systems(gabp_handle h, int nsys, const std::vector<int> &slots, const int *d_res,
                                   const double *d_rel, float ms, int *status_host, int *iters_host,
                                   double *relres_host) {
  h->prof.ms[PH_MULTI] += ms;
  std::vector<int> res(3 * nsys);
  std::vector<double> rel(nsys);
  GABP_CUDA(cudaMemcpyAsync(res.data(), d_res, sizeof(int) * 3 * nsys, cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaMemcpyAsync(rel.data(), d_rel, sizeof(double) * nsys, cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  int worst = GABP_OK;
  int64_t eu = 0, rmax = 0, steps = 0;
  for (int s = 0; s < nsys; ++s) {
    if (status_host) status_host[s] = res[s];
    if (iters_host) iters_host[s] = res[nsys + s];
    if (relres_host) relres_host[s] = rel[s];
    worst = std::max(worst, res[s]);
    eu += (int64_t)res[nsys + s] * slots[s];
    rmax = std::max<int64_t>(rmax, res[nsys + s]);
    steps = std::max<int64_t>(steps, res[2 * nsys + s]);
  }
  h->prof.rounds[PH_MULTI] += rmax;
  h->stats.rounds = rmax;
  h->stats.edge_updates = eu;
  h->stats.refine_steps = (int)steps;
  h->last_path = -1;
  return (gabp_status)worst;
}

}  // namespace gabp
