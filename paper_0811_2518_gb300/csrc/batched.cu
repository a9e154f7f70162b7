// batched.cu -- many right-hand sides in one launch sequence: FP32 mean messages
// for R right-hand sides sharing one converged precision state, FP64 iterative
// refinement per column.
//
// The precision messages depend on A only (eq_prec and eq_prec_message have no
// b in them), so the FP32 precision phase and the frozen coefficient pairs of
// solve32.cu serve every right-hand side.  The mean iteration is the recompute
// form of solve32.cu, run for RP columns at once:
//   h_{i->k}^{(t-1)} = c_out (h~_i^{(t-2)} - h_{k->i}^{(t-2)}),
//   h_{k->i}^{(t)}   = c_in  (h~_k^{(t-1)} - h_{i->k}^{(t-1)}).
// Layout: slot-major, column-minor -- H[e][r], NH[i][r] -- so a warp that owns a
// row reads one coefficient pair and one column index per slot (broadcast) and
// moves RP contiguous floats for the slot's messages and for the sender's
// aggregate: every edge-array access and every gather is a coalesced 128-512 B
// row.  One warp per row; lane l owns columns [l*VEC, l*VEC+VEC).
#include "gabp_internal.cuh"
#include "devutil.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace gabp {

namespace {

template <int VEC>
__device__ __forceinline__ void ldv(const float *p, float (&v)[VEC]) {
  if constexpr (VEC == 1) {
    v[0] = *p;
  } else if constexpr (VEC == 2) {
    const float2 q = *reinterpret_cast<const float2 *>(p);
    v[0] = q.x; v[1] = q.y;
  } else {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
}
template <int VEC>
__device__ __forceinline__ void ldv_cs(const float *p, float (&v)[VEC]) {
  if constexpr (VEC == 1) {
    v[0] = __ldcs(p);
  } else if constexpr (VEC == 2) {
    const float2 q = __ldcs(reinterpret_cast<const float2 *>(p));
    v[0] = q.x; v[1] = q.y;
  } else {
    const float4 q = __ldcs(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
}
template <int VEC>
__device__ __forceinline__ void stv(float *p, const float (&v)[VEC]) {
  if constexpr (VEC == 1) {
    *p = v[0];
  } else if constexpr (VEC == 2) {
    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
  } else {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
}
template <int VEC>
__device__ __forceinline__ void stv_cs(float *p, const float (&v)[VEC]) {
  if constexpr (VEC == 1) {
    __stcs(p, v[0]);
  } else if constexpr (VEC == 2) {
    __stcs(reinterpret_cast<float2 *>(p), make_float2(v[0], v[1]));
  } else {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
  }
}

struct ArgsB {
  int n, RP;
  const int *__restrict__ rp;
  const int *__restrict__ ci;
  const float2 *__restrict__ CF;
  const float *__restrict__ invP;
  float *H0, *H1;
  float *NH0, *NH1, *NH2;
  const float *rhs;
  DevCtl *ctl;
  double *red;  // [2][gridDim][RP] per-block per-column partial sums
  double *col;  // [4][RP] per-column results (0: dxx, 1: xx)
};

__device__ __forceinline__ float *ring3b(float *a, float *b, float *c, int t) {
  int m = t % 3;
  return m == 0 ? a : (m == 1 ? b : c);
}

// Per-column block reduction of NV per-thread vectors acc[j][v] (column l*VEC+v)
// over the block's warps, written to red[j][blockIdx][col].  Then the last block
// sums the columns over blocks into col[j][...].  Returns true in the last block.
template <int VEC, int NV>
__device__ bool col_reduce(const double (&acc)[NV][VEC], int RP, double *red, double *colout, unsigned int *arrive) {
  extern __shared__ double shc[];  // [NV][warps][RP]
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = kBlock / 32;
#pragma unroll
  for (int j = 0; j < NV; ++j)
#pragma unroll
    for (int v = 0; v < VEC; ++v) shc[(j * nw + w) * RP + l * VEC + v] = acc[j][v];
  __syncthreads();
  for (int c = threadIdx.x; c < NV * RP; c += kBlock) {
    const int j = c / RP, r = c % RP;
    double s = 0.0;
    for (int q = 0; q < nw; ++q) s += shc[(j * nw + q) * RP + r];
    red[((size_t)j * gridDim.x + blockIdx.x) * RP + r] = s;
  }
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(arrive, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  for (int c = threadIdx.x; c < NV * RP; c += kBlock) {
    const int j = c / RP, r = c % RP;
    double s = 0.0;
    for (int bI = 0; bI < (int)gridDim.x; ++bI) s += __ldcg(red + ((size_t)j * gridDim.x + bI) * RP + r);
    colout[j * RP + r] = s;
  }
  __threadfence();
  __syncthreads();
  return true;
}

// Round t of the batched frozen-precision mean iteration (one warp per row).
// Stops when every column with a nonzero iterate has ||dx_r|| <= inner_tol ||x_r||.
template <int VEC>
__global__ void __launch_bounds__(kBlock, 6) kb_mean(ArgsB a) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int t = ctl->round + 1;
  const int RP = a.RP;
  float *__restrict__ Hc = (t & 1) ? a.H1 : a.H0;  // holds t-2, becomes t
  const float *__restrict__ Hm1 = ring3b(a.NH0, a.NH1, a.NH2, t + 2);
  const float *__restrict__ Hm2 = ring3b(a.NH0, a.NH1, a.NH2, t + 1);
  float *__restrict__ Ht = ring3b(a.NH0, a.NH1, a.NH2, t);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  const int c0 = lane * VEC;
  float acc2[2][VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) acc2[0][v] = acc2[1][v] = 0.f;
  for (int i = warp; i < a.n; i += nwarps) {
    float hi2[VEC], acc[VEC];
    if (t >= 2) ldv<VEC>(Hm2 + (size_t)i * RP + c0, hi2);
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
    const int e0 = a.rp[i], e1 = a.rp[i + 1];
    int e = e0;
    for (; e + 1 < e1; e += 2) {  // two slots with their loads issued together
      const int k0 = a.ci[e], k1 = a.ci[e + 1];
      const float2 cf0 = a.CF[e], cf1 = a.CF[e + 1];
      float hs0[VEC], hs1[VEC], hk0[VEC], hk1[VEC], hn0[VEC], hn1[VEC];
      ldv_cs<VEC>(Hc + (size_t)e * RP + c0, hs0);
      ldv_cs<VEC>(Hc + (size_t)(e + 1) * RP + c0, hs1);
      ldv<VEC>(Hm1 + (size_t)k0 * RP + c0, hk0);
      ldv<VEC>(Hm1 + (size_t)k1 * RP + c0, hk1);
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        const float ho0 = t >= 2 ? cf0.y * (hi2[v] - hs0[v]) : 0.f;  // messages i -> k at t-1
        const float ho1 = t >= 2 ? cf1.y * (hi2[v] - hs1[v]) : 0.f;
        hn0[v] = cf0.x * (hk0[v] - ho0);                             // messages k -> i at t
        hn1[v] = cf1.x * (hk1[v] - ho1);
        acc[v] += hn0[v];
        acc[v] += hn1[v];
      }
      stv_cs<VEC>(Hc + (size_t)e * RP + c0, hn0);
      stv_cs<VEC>(Hc + (size_t)(e + 1) * RP + c0, hn1);
    }
    if (e < e1) {
      const int k = a.ci[e];
      const float2 cf = a.CF[e];
      float hs[VEC], hk[VEC];
      ldv_cs<VEC>(Hc + (size_t)e * RP + c0, hs);
      ldv<VEC>(Hm1 + (size_t)k * RP + c0, hk);
      float hn[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        const float hout = t >= 2 ? cf.y * (hi2[v] - hs[v]) : 0.f;  // message i -> k at t-1
        hn[v] = cf.x * (hk[v] - hout);                              // message k -> i at t
        acc[v] += hn[v];
      }
      stv_cs<VEC>(Hc + (size_t)e * RP + c0, hn);
    }
    float rh[VEC], hp[VEC], hnew[VEC];
    ldv<VEC>(a.rhs + (size_t)i * RP + c0, rh);
    ldv<VEC>(Hm1 + (size_t)i * RP + c0, hp);
    const float ip = a.invP[i];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      hnew[v] = rh[v] + acc[v];
      const float x = hnew[v] * ip, dx = (hnew[v] - hp[v]) * ip;
      acc2[0][v] = fmaf(dx, dx, acc2[0][v]);
      acc2[1][v] = fmaf(x, x, acc2[1][v]);
    }
    stv<VEC>(Ht + (size_t)i * RP + c0, hnew);
  }
  double accd[2][VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    accd[0][v] = (double)acc2[0][v];
    accd[1][v] = (double)acc2[1][v];
  }
  if (col_reduce<VEC, 2>(accd, RP, a.red, a.col, &ctl->arrive) && threadIdx.x == 0) {
    ctl->round = t;
    int notdone = 0;
    bool finite = true;
    for (int r = 0; r < RP; ++r) {
      const double dxx = a.col[r], xx = a.col[RP + r];
      if (!isfinite(dxx) || !isfinite(xx)) finite = false;
      if (xx > 0.0 && !(dxx <= ctl->tol2bb * xx)) ++notdone;
    }
    ctl->rr = (double)notdone;
    if (ctl->no_stop) {
    } else if (!finite) {
      ctl->status = GABP_DIVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (t >= 2 && notdone == 0) {
      ctl->status = GABP_OK; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    } else if (t >= ctl->max_iter) {
      ctl->status = GABP_NOT_CONVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
    }
    ctl->arrive = 0;
    __threadfence();
  }
}

// R = B - A X in FP64 for all columns (one warp per row, full CSR with the
// diagonal); FP32 copies seed the next inner solve; per-column ||r||^2.
template <int VEC>
__global__ void __launch_bounds__(kBlock) kb_residual(int n, int RP, const int *__restrict__ rowptr,
                                                     const int *__restrict__ col, const double *__restrict__ val,
                                                     const double *__restrict__ Bt, const double *__restrict__ X,
                                                     float *__restrict__ rhs, float *__restrict__ nh0, double *red,
                                                     double *colout, unsigned int *arrive) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  const int c0 = lane * VEC;
  double rrd[1][VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) rrd[0][v] = 0.0;
  for (int i = warp; i < n; i += nwarps) {
    double ax[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) ax[v] = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const double A = val[p];
      const double *xr = X + (size_t)col[p] * RP + c0;
#pragma unroll
      for (int v = 0; v < VEC; ++v) ax[v] = fma(A, xr[v], ax[v]);
    }
    float rf[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const double r = Bt[(size_t)i * RP + c0 + v] - ax[v];
      rrd[0][v] = fma(r, r, rrd[0][v]);
      rf[v] = (float)r;
    }
    stv<VEC>(rhs + (size_t)i * RP + c0, rf);
    stv<VEC>(nh0 + (size_t)i * RP + c0, rf);
  }
  if (col_reduce<VEC, 1>(rrd, RP, red, colout, arrive) && threadIdx.x == 0) {
    *arrive = 0;  // colout[r] now holds column r's ||b_r - A x_r||^2
    __threadfence();
  }
}

// X[i][r] += h~_i^{(T)}[r] / P~_i
template <int VEC>
__global__ void kb_update(int n, int RP, double *__restrict__ X, const float *__restrict__ hT,
                          const float *__restrict__ invP) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < n; i += nwarps) {
    const float ip = invP[i];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const size_t q = (size_t)i * RP + lane * VEC + v;
      X[q] += (double)(hT[q] * ip);
    }
  }
}

// Column-major user arrays <-> row-major [n][RP] work arrays (32 x 32 tiles).
__global__ void kb_gather_cols(int n, int R, int RP, const double *__restrict__ B, int64_t ld,
                               double *__restrict__ Bt) {
  __shared__ double tile[32][33];
  const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int r = r0 + q, i = i0 + threadIdx.x;
    tile[q][threadIdx.x] = (r < R && i < n) ? B[(size_t)r * ld + i] : 0.0;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int i = i0 + q, r = r0 + threadIdx.x;
    if (i < n && r < RP) Bt[(size_t)i * RP + r] = tile[threadIdx.x][q];
  }
}

__global__ void kb_scatter_cols(int n, int R, int RP, const double *__restrict__ Xt, double *__restrict__ X,
                                int64_t ld) {
  __shared__ double tile[32][33];
  const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int i = i0 + q, r = r0 + threadIdx.x;
    tile[q][threadIdx.x] = (i < n && r < RP) ? Xt[(size_t)i * RP + r] : 0.0;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int r = r0 + q, i = i0 + threadIdx.x;
    if (r < R && i < n) X[(size_t)r * ld + i] = tile[threadIdx.x][q];
  }
}

// ---------------------------------------------------------------------------- serial schedule, R right-hand sides
// Pass c of a serial frozen-coefficient mean sweep for RP columns (one warp per
// new row, lane l owns columns [l*VEC, l*VEC+VEC)); the layout, the order and
// the recompute identity are those of serial.cu.  Per-column sums of the pass
// go to acc[2][RP]; after the last pass every column with a nonzero iterate must
// have its estimated error (step x q/(1-q), q the step ratio of the last two
// sweeps, taken between 1 and 4 steps) within itol ||x_r||.
struct ArgsBS {
  int n, C, RP;
  const int *__restrict__ co;
  const int *__restrict__ sci;
  const int *__restrict__ scol;
  const int *__restrict__ srp;
  const float2 *__restrict__ sCF;
  const float *__restrict__ sinvP;
  const float *__restrict__ srhs;  // [n][RP] new order
  float *sH;                       // [E][RP] serial slot order
  float *hfire;                    // [n][RP] new order
  DevCtl *ctl;
  double *red;
  double *col;                     // [2][RP] pass sums, then [2][RP] sweep sums, [RP] previous step
};

#ifndef GABP_KBS_U
#define GABP_KBS_U 3
#endif
#ifndef GABP_KBS_MINB
#define GABP_KBS_MINB 6
#endif
constexpr int kBsU = GABP_KBS_U;  // slots of a row whose loads are issued together

template <int VEC>
__global__ void __launch_bounds__(kBlock, GABP_KBS_MINB) kbs_pass(ArgsBS a, int c, int skip0, int skipn) {
  DevCtl *ctl = a.ctl;
  if (ctl->done) return;
  const int RP = a.RP;
  const int cn = c + 1 == a.C ? 0 : c + 1;
  const int nv = a.n - skipn;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  const int c0 = lane * VEC;
  float acc2[2][VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) acc2[0][v] = acc2[1][v] = 0.f;
  for (int vr = warp; vr < nv; vr += nwarps) {
    const int j = vr < skip0 ? vr : vr + skipn;
    float hj[VEC], acc[VEC];
    ldv<VEC>(a.hfire + (size_t)j * RP + c0, hj);
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
    const int s0 = a.co[(size_t)c * a.n + j], s1 = a.co[(size_t)(c + 1) * a.n + j];
    int e = s0;
    for (; e + kBsU <= s1; e += kBsU) {  // kBsU slots with their loads issued together
      int k[kBsU];
      float2 cf[kBsU];
      float hs[kBsU][VEC], hk[kBsU][VEC];
#pragma unroll
      for (int u = 0; u < kBsU; ++u) {
        k[u] = a.sci[e + u];
        cf[u] = a.sCF[e + u];
      }
#pragma unroll
      for (int u = 0; u < kBsU; ++u) {
        ldv_cs<VEC>(a.sH + (size_t)(e + u) * RP + c0, hs[u]);
        ldv<VEC>(a.hfire + (size_t)k[u] * RP + c0, hk[u]);
      }
#pragma unroll
      for (int u = 0; u < kBsU; ++u) {
        float hn[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          hn[v] = cf[u].x * (hk[u][v] - cf[u].y * (hj[v] - hs[u][v]));  // message k -> j, k firing now
          acc[v] += hn[v];                                              // (reverse message recomputed)
        }
        stv_cs<VEC>(a.sH + (size_t)(e + u) * RP + c0, hn);
      }
    }
    for (; e < s1; ++e) {
      const int k = a.sci[e];
      const float2 cf = a.sCF[e];
      float hs[VEC], hk[VEC], hn[VEC];
      ldv_cs<VEC>(a.sH + (size_t)e * RP + c0, hs);
      ldv<VEC>(a.hfire + (size_t)k * RP + c0, hk);
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        const float hout = cf.y * (hj[v] - hs[v]);  // message j -> k when j last fired
        hn[v] = cf.x * (hk[v] - hout);              // message k -> j, k firing now
        acc[v] += hn[v];
      }
      stv_cs<VEC>(a.sH + (size_t)e * RP + c0, hn);
    }
    if (a.scol[j] == cn) {  // j fires next: its aggregate over the whole row
      for (int e = a.srp[j]; e < s0; ++e) {
        float hs[VEC];
        ldv<VEC>(a.sH + (size_t)e * RP + c0, hs);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] += hs[v];
      }
      for (int e = s1; e < a.srp[j + 1]; ++e) {
        float hs[VEC];
        ldv<VEC>(a.sH + (size_t)e * RP + c0, hs);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] += hs[v];
      }
      float rh[VEC], hnew[VEC];
      ldv<VEC>(a.srhs + (size_t)j * RP + c0, rh);
      const float ip = a.sinvP[j];
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        hnew[v] = rh[v] + acc[v];
        const float x = hnew[v] * ip, dx = (hnew[v] - hj[v]) * ip;
        acc2[0][v] = fmaf(dx, dx, acc2[0][v]);
        acc2[1][v] = fmaf(x, x, acc2[1][v]);
      }
      stv<VEC>(a.hfire + (size_t)j * RP + c0, hnew);
    }
  }
  double accd[2][VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    accd[0][v] = (double)acc2[0][v];
    accd[1][v] = (double)acc2[1][v];
  }
  if (col_reduce<VEC, 2>(accd, RP, a.red, a.col, &ctl->arrive)) {
    // the last block: add the pass to the sweep's per-column sums
    double *sw = a.col + 2 * RP, *prev = a.col + 4 * RP;
    for (int r = threadIdx.x; r < 2 * RP; r += kBlock) sw[r] += a.col[r];
    __syncthreads();
    if (threadIdx.x == 0) {
      if (c == a.C - 1) {  // the sweep is complete: per-column decision
        const int t = ctl->round + 1;
        ctl->round = t;
        int notdone = 0;
        bool finite = true;
        for (int r = 0; r < RP; ++r) {
          const double dd = sw[r], xx = sw[RP + r], pv = prev[r];
          if (!isfinite(dd) || !isfinite(xx)) finite = false;
          double f2 = 1.0;
          if (t >= 3 && pv > 0.0) {
            const double q = sqrt(dd / pv);
            f2 = q < 0.8 ? fmax(1.0, (q / (1.0 - q)) * (q / (1.0 - q))) : 16.0;
          }
          if (xx > 0.0 && !(dd * f2 <= ctl->tol2bb * xx)) ++notdone;
          prev[r] = dd;
          sw[r] = 0.0;
          sw[RP + r] = 0.0;
        }
        ctl->rr = (double)notdone;
        if (!finite) {
          ctl->status = GABP_DIVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
        } else if (t >= 2 && notdone == 0) {
          ctl->status = GABP_OK; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
        } else if (t >= ctl->max_iter) {
          ctl->status = GABP_NOT_CONVERGED; ctl->iters = t; ctl->result_round = t; ctl->done = 1;
        }
      }
      ctl->arrive = 0;
      __threadfence();
    }
  }
}

// new-order rows of an [n][RP] FP32 array from the input order; the inner
// solve starts with h~ = r
__global__ void kbs_init(int n, int RP, const int *__restrict__ oid, const float *__restrict__ rhs,
                         float *__restrict__ srhs, float *__restrict__ hfire) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < n; j += nwarps) {
    const size_t src = (size_t)oid[j] * RP, dst = (size_t)j * RP;
    for (int r = lane; r < RP; r += 32) {
      const float v = rhs[src + r];
      srhs[dst + r] = v;
      hfire[dst + r] = v;
    }
  }
}

// X[oid[j]][r] += h~_j^fire[r] / P~_j
__global__ void kbs_update(int n, int RP, const int *__restrict__ oid, const float *__restrict__ hfire,
                           const float *__restrict__ sinvP, double *__restrict__ X) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < n; j += nwarps) {
    const float ip = sinvP[j];
    const size_t src = (size_t)j * RP, dst = (size_t)oid[j] * RP;
    for (int r = lane; r < RP; r += 32) X[dst + r] += (double)(hfire[src + r] * ip);
  }
}

__global__ void kbs_ctl_reset(DevCtl *c, int max_iter, double tol2, double *col, int RP) {
  c->round = 0;
  c->done = 0;
  c->status = GABP_NOT_CONVERGED;
  c->iters = 0;
  c->result_round = 0;
  c->max_iter = max_iter;
  c->tol2bb = tol2;
  c->arrive = 0;
  c->no_stop = 0;
  for (int r = 2 * RP; r < 5 * RP; ++r) col[r] = 0.0;  // sweep sums and previous steps
}

__global__ void kb_ctl_reset(DevCtl *c, int max_iter, double tol2) {
  c->round = 0;
  c->done = 0;
  c->status = GABP_NOT_CONVERGED;
  c->iters = 0;
  c->result_round = 0;
  c->max_iter = max_iter;
  c->check_from = 1;
  c->stable = 0;
  c->tol2bb = tol2;
  c->arrive = 0;
  c->no_stop = 0;
}

}  // namespace

struct WorkB {
  int RP = 0;
  float *H[2] = {nullptr, nullptr};
  float *NH[3] = {nullptr, nullptr, nullptr};
  float *rhs = nullptr;
  double *X = nullptr, *Bt = nullptr;
  double *red = nullptr, *col = nullptr;
  unsigned int *arrive = nullptr;
  cudaGraphExec_t graph = nullptr;
  long long graph_key = -1;
  float *sH = nullptr, *hfire = nullptr, *srhs = nullptr;  // serial schedule: [E][RP], [n][RP], [n][RP]
  cudaGraphExec_t sgraph = nullptr;
  long long sgraph_key = -1;
};

void free_wb(gabp_handle h) {
  WorkB *w = h->wb;
  if (!w) return;
  cudaFree(w->H[0]); cudaFree(w->H[1]);
  for (int j = 0; j < 3; ++j) cudaFree(w->NH[j]);
  cudaFree(w->rhs); cudaFree(w->X); cudaFree(w->Bt); cudaFree(w->red); cudaFree(w->col); cudaFree(w->arrive);
  cudaFree(w->sH); cudaFree(w->hfire); cudaFree(w->srhs);
  if (w->graph) cudaGraphExecDestroy(w->graph);
  if (w->sgraph) cudaGraphExecDestroy(w->sgraph);
  delete w;
  h->wb = nullptr;
}

static gabp_status ensure_wb(gabp_handle h, int RP) {
  if (h->wb && h->wb->RP == RP) return GABP_OK;
  free_wb(h);
  h->wb = new WorkB();
  WorkB *w = h->wb;
  const size_t E = (size_t)(h->g.E > 0 ? h->g.E : 1), n = (size_t)h->g.n;
  GABP_CUDA(cudaMalloc(&w->H[0], sizeof(float) * E * RP));
  GABP_CUDA(cudaMalloc(&w->H[1], sizeof(float) * E * RP));
  for (int j = 0; j < 3; ++j) GABP_CUDA(cudaMalloc(&w->NH[j], sizeof(float) * n * RP));
  GABP_CUDA(cudaMalloc(&w->rhs, sizeof(float) * n * RP));
  GABP_CUDA(cudaMalloc(&w->X, sizeof(double) * n * RP));
  GABP_CUDA(cudaMalloc(&w->Bt, sizeof(double) * n * RP));
  GABP_CUDA(cudaMalloc(&w->red, sizeof(double) * 2 * (size_t)h->max_blocks * RP));
  GABP_CUDA(cudaMalloc(&w->col, sizeof(double) * 5 * RP));
  GABP_CUDA(cudaMalloc(&w->arrive, sizeof(unsigned int)));
  GABP_CUDA(cudaMemsetAsync(w->arrive, 0, sizeof(unsigned int), h->stream));
  w->RP = RP;
  return GABP_OK;
}

template <int VEC>
static gabp_status batched_chunk(gabp_handle h, int R, const double *B, double *X, int64_t ld, double tol,
                                 int max_iter, int *iters, double *relres_host, int *worst) {
  constexpr int RP = 32 * VEC;
  gabp_status s = ensure_wb(h, RP);
  if (s != GABP_OK) return s;
  WorkB &w = *h->wb;
  Graph &g = h->g;
  Work32 &w32 = h->w32;
  const size_t E = (size_t)(g.E > 0 ? g.E : 1);
  const size_t shmem = sizeof(double) * 2 * (kBlock / 32) * RP;
  // a full wave of one-warp-per-row blocks
  auto grid_of = [&](auto kern) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kBlock, shmem) != cudaSuccess || nb < 1) {
      cudaGetLastError();
      nb = 1;
    }
    return blocks_for(g.n, kBlock / 32, nb * h->num_sms);
  };
  const int nb_mean = grid_of(kb_mean<VEC>);
  const int nb_res = grid_of(kb_residual<VEC>);
  dim3 tb(32, 8), tg((g.n + 31) / 32, RP / 32);
  kb_gather_cols<<<tg, tb, 0, h->stream>>>(g.n, R, RP, B, ld, w.Bt);
  GABP_CUDA(cudaMemsetAsync(w.X, 0, sizeof(double) * g.n * RP, h->stream));
  kb_residual<VEC><<<nb_res, kBlock, shmem, h->stream>>>(g.n, RP, g.rowptr, g.col, g.val, w.Bt, w.X, w.rhs, w.NH[0],
                                                         w.red, w.col, w.arrive);
  h->prof.launches += 2;
  GABP_CUDA(cudaGetLastError());
  std::vector<double> colh(4 * RP);
  auto read_cols = [&]() -> gabp_status {
    GABP_CUDA(cudaMemcpyAsync(colh.data(), w.col, sizeof(double) * RP, cudaMemcpyDeviceToHost, h->stream));
    GABP_CUDA(cudaStreamSynchronize(h->stream));
    return GABP_OK;
  };
  if ((s = read_cols()) != GABP_OK) return s;
  std::vector<double> bb(R), rr(R);
  for (int r = 0; r < R; ++r) bb[r] = rr[r] = colh[r];
  ArgsB a;
  a.n = g.n; a.RP = RP; a.rp = g.rp; a.ci = g.ci; a.CF = w32.CF; a.invP = w32.invP;
  a.H0 = w.H[0]; a.H1 = w.H[1]; a.NH0 = w.NH[0]; a.NH1 = w.NH[1]; a.NH2 = w.NH[2];
  a.rhs = w.rhs; a.ctl = h->ctl; a.red = w.red; a.col = w.col;
  const double itol = h->opt.inner_tol;
  const bool serial = h->opt.schedule == 1;
  ArgsBS as;
  int nb_ser = 1;
  if (serial) {
    if ((s = serial_freeze32(h, w32.CF, w32.invP)) != GABP_OK) return s;
    WorkS &ws = h->ws;
    if (!w.sH) {
      GABP_CUDA(cudaMalloc(&w.sH, sizeof(float) * E * RP));
      GABP_CUDA(cudaMalloc(&w.hfire, sizeof(float) * g.n * RP));
      GABP_CUDA(cudaMalloc(&w.srhs, sizeof(float) * g.n * RP));
    }
    as.n = g.n; as.C = ws.C; as.RP = RP; as.co = ws.co; as.sci = ws.sci; as.scol = ws.scol; as.srp = ws.srp;
    as.sCF = ws.sCF; as.sinvP = ws.sinvP; as.srhs = w.srhs; as.sH = w.sH; as.hfire = w.hfire;
    as.ctl = h->ctl; as.red = w.red; as.col = w.col;
    nb_ser = grid_of(kbs_pass<VEC>);
  }
  int total_inner = 0;
  auto all_done = [&]() {
    for (int r = 0; r < R; ++r)
      if (bb[r] > 0.0 && !(rr[r] <= tol * tol * bb[r])) return false;
    return true;
  };
  bool diverged = false;
  for (int step = 0; step < h->opt.max_refine && !all_done() && total_inner < max_iter; ++step) {
    GABP_CUDA(cudaMemsetAsync(serial ? w.sH : w.H[0], 0, sizeof(float) * E * RP, h->stream));
    const int cap = std::min(h->opt.inner_max_iter, std::max(1, max_iter - total_inner));
    double worst_ratio = 0.0;  // the column furthest from its target sets the inner tolerance
    for (int r = 0; r < R; ++r)
      if (bb[r] > 0.0) worst_ratio = std::max(worst_ratio, rr[r] / bb[r]);
    const double it_tol = inner_target(itol, tol, 1.0, worst_ratio);
    if (serial) {
      WorkS &ws = h->ws;
      kbs_init<<<std::max(1, (g.n + 7) / 8), kBlock, 0, h->stream>>>(g.n, RP, ws.oid, w.rhs, w.srhs, w.hfire);
      kbs_ctl_reset<<<1, 1, 0, h->stream>>>(h->ctl, cap, it_tol * it_tol, w.col, RP);
      h->prof.launches += 2;
      GABP_CUDA(cudaGetLastError());
      s = run_rounds(h, &w.sgraph, &w.sgraph_key, RP | (ws.C << 16), [&] {
        for (int c = 0; c < ws.C; ++c)
          kbs_pass<VEC><<<nb_ser, kBlock, shmem, h->stream>>>(as, c, ws.cstart[c], ws.cstart[c + 1] - ws.cstart[c]);
      }, cap, PH_MEAN32);
    } else {
      kb_ctl_reset<<<1, 1, 0, h->stream>>>(h->ctl, cap, it_tol * it_tol);
      h->prof.launches += 1;
      GABP_CUDA(cudaGetLastError());
      s = run_rounds(h, &w.graph, &w.graph_key, RP, [&] { kb_mean<VEC><<<nb_mean, kBlock, shmem, h->stream>>>(a); },
                     cap, PH_MEAN32);
    }
    if (s != GABP_OK) return s;
    const DevCtl c = *h->ctl_host;
    total_inner += c.round;
    h->stats.rounds += c.round;
    h->stats.edge_updates += (int64_t)c.round * g.E * R;
    if (c.status == GABP_DIVERGED) { diverged = true; break; }
    float *hT = w.NH[c.result_round % 3];
    prof_begin(h);
    if (serial)
      kbs_update<<<std::max(1, (g.n + 7) / 8), kBlock, 0, h->stream>>>(g.n, RP, h->ws.oid, w.hfire, h->ws.sinvP, w.X);
    else
      kb_update<VEC><<<std::max(1, (g.n + 7) / 8), kBlock, 0, h->stream>>>(g.n, RP, w.X, hT, w32.invP);
    kb_residual<VEC><<<nb_res, kBlock, shmem, h->stream>>>(g.n, RP, g.rowptr, g.col, g.val, w.Bt, w.X, w.rhs,
                                                           w.NH[0], w.red, w.col, w.arrive);
    prof_end(h);
    h->prof.launches += 2;
    GABP_CUDA(cudaGetLastError());
    if ((s = read_cols()) != GABP_OK) return s;
    prof_collect(h, PH_REFINE64, 1);
    h->stats.refine_steps += 1;
    for (int r = 0; r < R; ++r) {
      rr[r] = colh[r];
      if (!std::isfinite(rr[r])) diverged = true;
    }
    if (diverged) break;
  }
  dim3 sg((g.n + 31) / 32, RP / 32);
  kb_scatter_cols<<<sg, tb, 0, h->stream>>>(g.n, R, RP, w.X, X, ld);
  h->prof.launches += 1;
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  int st = GABP_OK;
  for (int r = 0; r < R; ++r) {
    const double rel = bb[r] > 0.0 ? std::sqrt(rr[r] / bb[r]) : 0.0;
    if (relres_host) relres_host[r] = rel;
    if (diverged) st = std::max(st, (int)GABP_DIVERGED);
    else if (bb[r] > 0.0 && !(rr[r] <= tol * tol * bb[r])) st = std::max(st, (int)GABP_NOT_CONVERGED);
  }
  *worst = std::max(*worst, st);
  *iters += total_inner;
  return GABP_OK;
}

gabp_status solve_batched32(gabp_handle h, int nrhs, const double *B, double *X, int64_t ld, double tol,
                            int max_iter, int *iters, double *relres_host) {
  NvtxRange nvtx_("gabp batched right-hand sides");
  if (nrhs < 1 || ld < h->g.n) return GABP_ERR_INVALID;
  gabp_status s = ensure_w32(h, 1);
  if (s != GABP_OK) return s;
  h->stats.rounds = 0;
  h->stats.edge_updates = 0;
  h->stats.refine_steps = 0;
  if (!h->w32.coef_ready || !h->opt.reuse_precisions) {
    h->w32.coef_ready = false;
    if ((s = precision_phase32(h, nullptr)) != GABP_OK) return s;
    h->stats.edge_updates += h->stats.rounds * (int64_t)h->g.E;  // precision rounds serve every column
  }
  int worst = GABP_OK, total = 0;
  for (int r0 = 0; r0 < nrhs; r0 += 128) {
    const int R = std::min(128, nrhs - r0);
    const double *Bc = B + (size_t)r0 * ld;
    double *Xc = X + (size_t)r0 * ld;
    double *rel = relres_host ? relres_host + r0 : nullptr;
    if (R <= 32) s = batched_chunk<1>(h, R, Bc, Xc, ld, tol, max_iter, &total, rel, &worst);
    else if (R <= 64) s = batched_chunk<2>(h, R, Bc, Xc, ld, tol, max_iter, &total, rel, &worst);
    else s = batched_chunk<4>(h, R, Bc, Xc, ld, tol, max_iter, &total, rel, &worst);
    if (s != GABP_OK) return s;
  }
  if (iters) *iters = total;
  h->last_path = 1;
  return (gabp_status)worst;
}

}  // namespace gabp
