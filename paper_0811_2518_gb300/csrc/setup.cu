// setup.cu -- gabp_create / gabp_destroy: validation of A, the off-diagonal
// receiver-layout CSR, the diagonal, and the reverse-edge index.
//
// The graph of A: one node per variable, one undirected edge per nonzero
// off-diagonal pair, N(i) excluding i itself (paper, Sec. "From Linear Algebra
// to Probabilistic Inference"; Algorithm 1, step 1, "set the neighborhood").
// Every directed edge k -> i is a slot of row i; the broadcast form
// (Algorithm 2) needs, for each slot, the slot of the reverse edge: rev[].
#include "gabp_internal.cuh"

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

namespace gabp {

static thread_local std::string g_last_error;

void set_last_error(const std::string &s) { g_last_error = s; }

gabp_status cuda_fail(cudaError_t e, const char *what) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  g_last_error = buf;
  cudaGetLastError();  // a failed call's error is reported here, not again by a later check
  if (e == cudaErrorMemoryAllocation) return GABP_ERR_NOMEM;
  return GABP_ERR_CUDA;
}

enum : int {
  BAD_ROWPTR = 1,
  BAD_COL = 2,
  BAD_DIAG = 4,
  BAD_OFFDIAG = 8,
  BAD_PATTERN = 16,
  BAD_VALUE = 32,
};

// rowptr must start at 0, end at nnz and never decrease.
__global__ void k_check_rowptr(int n, int64_t nnz, const int *__restrict__ rowptr, int *flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = rowptr[i], b = rowptr[i + 1];
  bool bad = a > b || a < 0 || (int64_t)b > nnz;
  if (i == 0 && a != 0) bad = true;
  if (i == n - 1 && (int64_t)b != nnz) bad = true;
  if (bad) atomicOr(flag, BAD_ROWPTR);
}

// Columns in range and strictly increasing, exactly one nonzero finite diagonal,
// nonzero finite off-diagonals.  dpos[i] = position of the diagonal in row i.
__global__ void k_check_rows(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                             const double *__restrict__ val, int *__restrict__ dpos, int *flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = rowptr[i], b = rowptr[i + 1];
  int nd = 0, pos = -1, prev = -1, f = 0;
  for (int p = a; p < b; ++p) {
    int c = col[p];
    double v = val[p];
    if (c < 0 || c >= n || c <= prev) f |= BAD_COL;
    prev = c;
    if (c == i) {
      ++nd;
      pos = p - a;
      if (v == 0.0 || !isfinite(v)) f |= BAD_DIAG;
    } else if (v == 0.0 || !isfinite(v)) {
      f |= BAD_OFFDIAG;
    }
  }
  if (nd != 1) f |= BAD_DIAG;
  dpos[i] = pos < 0 ? 0 : pos;
  if (f) atomicOr(flag, f);
}

// Split off the diagonal: off-diagonal row i starts at rowptr[i] - i.
__global__ void k_compact(int n, const int *__restrict__ rowptr, const int *__restrict__ col,
                          const double *__restrict__ val, const int *__restrict__ dpos, int *__restrict__ rp,
                          int *__restrict__ ci, double *__restrict__ av, double *__restrict__ ad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) {
    rp[n] = rowptr[n] - n;
    return;
  }
  int a = rowptr[i], b = rowptr[i + 1], d = dpos[i];
  int e0 = a - i;
  rp[i] = e0;
  ad[i] = val[a + d];
  for (int q = 0; q < b - a; ++q) {
    if (q == d) continue;
    int e = e0 + (q < d ? q : q - 1);
    ci[e] = col[a + q];
    av[e] = val[a + q];
  }
}

// New values on the existing pattern: A_ik == A_ki bit for bit through rev[].
__global__ void k_values_to_f32(int64_t E, const double *__restrict__ s, float *__restrict__ d) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < E) d[e] = (float)s[e];
}

__global__ void k_check_sym(int64_t E, const double *__restrict__ av, const int *__restrict__ rev, int *flag) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < E && __double_as_longlong(av[e]) != __double_as_longlong(av[rev[e]])) atomicOr(flag, (int)BAD_VALUE);
}

// rev[e] for slot e = (row i, column k): binary search of i among row k's columns.
// The pattern and the values must be symmetric bit for bit.
__global__ void k_rev(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ av,
                      int *__restrict__ rev, int *flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = 0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    int k = ci[e];
    int lo = rp[k], hi = rp[k + 1] - 1, hit = -1;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1;
      int c = ci[mid];
      if (c == i) { hit = mid; break; }
      if (c < i) lo = mid + 1; else hi = mid - 1;
    }
    if (hit < 0) {
      f |= BAD_PATTERN;
      rev[e] = e;  // keeps every later access in bounds; the handle is rejected anyway
    } else {
      rev[e] = hit;
      if (__double_as_longlong(av[hit]) != __double_as_longlong(av[e])) f |= BAD_VALUE;
    }
  }
  if (f) atomicOr(flag, f);
}

static void free_graph(Graph &g) {
  cudaFree(g.rowptr); cudaFree(g.col); cudaFree(g.val);
  cudaFree(g.rp); cudaFree(g.ci); cudaFree(g.rev); cudaFree(g.dpos);
  cudaFree(g.av); cudaFree(g.ad); cudaFree(g.av32); cudaFree(g.ad32);
  g = Graph{};
}

__global__ void k_ctl_arm_tune(DevCtl *c, const double *b) {
  c->round = 0;
  c->done = 0;
  c->status = GABP_NOT_CONVERGED;
  c->max_iter = 0x7fffffff;
  c->check_from = 1;
  c->stable = 0;
  c->tol2bb = -1.0;
  c->arrive = 0;
  c->edge_bad = 0;
  c->b = b;
  c->no_stop = 1;
  c->hist = nullptr;  // tuning rounds record no residual history
  c->hist_cap = 0;
  c->hist_len = 0;
}

gabp_status tune_ctl(gabp_handle h, const double *b) {
  if (!h->ctl_tune) {
    GABP_CUDA(cudaMalloc(&h->ctl_tune, sizeof(DevCtl)));
    GABP_CUDA(cudaMemsetAsync(h->ctl_tune, 0, sizeof(DevCtl), h->stream));
  }
  if (!h->ctl_tune) return GABP_ERR_NOMEM;
  k_ctl_arm_tune<<<1, 1, 0, h->stream>>>(h->ctl_tune, b ? b : h->g.ad);
  GABP_CUDA(cudaGetLastError());
  return GABP_OK;
}

gabp_status read_ctl(gabp_handle h) {
  GABP_CUDA(cudaMemcpyAsync(h->ctl_host, h->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return GABP_OK;
}

static gabp_status destroy_impl(gabp_handle h) {
  if (!h) return GABP_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->g64) cudaGraphExecDestroy(h->g64);
  if (h->gP32) cudaGraphExecDestroy(h->gP32);
  if (h->gH32) cudaGraphExecDestroy(h->gH32);
  if (h->gJ32) cudaGraphExecDestroy(h->gJ32);
  if (h->gRef) cudaGraphExecDestroy(h->gRef);
  if (h->gRefG) cudaGraphDestroy(h->gRefG);
  free_w64(h);
  free_w32(h);
  free_wb(h);
  free_ws(h);
  free_wf(h);
  free_gsell(h);
  free_graph(h->g);
  cudaFree(h->ctl);
  cudaFreeHost(h->ctl_host);
  cudaFree(h->partials);
  cudaFree(h->hb);
  cudaFree(h->hx);
  cudaFree(h->gamma);
  cudaFree(h->hist);
  if (h->own_stream) {
    cudaStreamSynchronize(h->own_stream);
    cudaStreamDestroy(h->own_stream);
  }
  if (h->caller_ev) cudaEventDestroy(h->caller_ev);
  cudaFree(h->ig_buf);
  cudaFree(h->ctl_tune);
  cudaFree(h->lsq_b);
  cudaFree(h->lsq_x);
  if (h->prof.e0) cudaEventDestroy(h->prof.e0);
  if (h->prof.e1) cudaEventDestroy(h->prof.e1);
  cudaSetDevice(cur);
  delete h;
  return GABP_OK;
}

static gabp_status create_impl(gabp_handle h, int n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                               const double *val, int mem_space) {
  Graph &g = h->g;
  g.n = n;
  g.nnz = nnz;
  order_after_caller(h);  // a device CSR may still be in flight on the caller's default stream
  GABP_CUDA(cudaMalloc(&g.rowptr, sizeof(int) * (n + 1)));
  GABP_CUDA(cudaMalloc(&g.col, sizeof(int) * nnz));
  GABP_CUDA(cudaMalloc(&g.val, sizeof(double) * nnz));
  GABP_CUDA(cudaMalloc(&g.dpos, sizeof(int) * n));
  cudaMemcpyKind kind = mem_space == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  GABP_CUDA(cudaMemcpyAsync(g.rowptr, rowptr, sizeof(int) * (n + 1), kind, h->stream));
  GABP_CUDA(cudaMemcpyAsync(g.col, col, sizeof(int) * nnz, kind, h->stream));
  GABP_CUDA(cudaMemcpyAsync(g.val, val, sizeof(double) * nnz, kind, h->stream));

  int *dflag = nullptr;
  GABP_CUDA(cudaMalloc(&dflag, sizeof(int)));
  int hflag = 0;
  auto fail = [&](gabp_status s) { cudaFree(dflag); return s; };
  auto read_flag = [&]() -> gabp_status {
    cudaError_t e = cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "validation read-back");
    return GABP_OK;
  };
  if (cudaMemsetAsync(dflag, 0, sizeof(int), h->stream) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "memset"));
  int nb = (n + kBlock - 1) / kBlock;
  k_check_rowptr<<<nb, kBlock, 0, h->stream>>>(n, nnz, g.rowptr, dflag);
  gabp_status s = read_flag();
  if (s != GABP_OK) return fail(s);
  if (hflag) {
    set_last_error("gabp_create: rowptr is not a valid CSR row pointer");
    return fail(GABP_ERR_INVALID);
  }
  k_check_rows<<<nb, kBlock, 0, h->stream>>>(n, g.rowptr, g.col, g.val, g.dpos, dflag);
  if ((s = read_flag()) != GABP_OK) return fail(s);
  if (hflag) {
    set_last_error(hflag & BAD_COL    ? "gabp_create: column index out of range or not strictly increasing"
                 : hflag & BAD_DIAG   ? "gabp_create: a row lacks a single nonzero finite diagonal entry"
                                      : "gabp_create: zero or non-finite off-diagonal entry");
    return fail(GABP_ERR_INVALID);
  }
  int64_t E = nnz - n;
  if (E < 0 || E >= INT32_MAX) return fail(GABP_ERR_INVALID);
  g.E = (int)E;
  size_t Ea = (size_t)(E > 0 ? E : 1);
  if (cudaMalloc(&g.rp, sizeof(int) * (n + 1)) != cudaSuccess || cudaMalloc(&g.ci, sizeof(int) * Ea) != cudaSuccess ||
      cudaMalloc(&g.rev, sizeof(int) * Ea) != cudaSuccess || cudaMalloc(&g.av, sizeof(double) * Ea) != cudaSuccess ||
      cudaMalloc(&g.ad, sizeof(double) * n) != cudaSuccess)
    return fail(cuda_fail(cudaErrorMemoryAllocation, "gabp_create graph arrays"));
  k_compact<<<(n + 1 + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(n, g.rowptr, g.col, g.val, g.dpos, g.rp, g.ci,
                                                                      g.av, g.ad);
  k_rev<<<nb, kBlock, 0, h->stream>>>(n, g.rp, g.ci, g.av, g.rev, dflag);
  if ((s = read_flag()) != GABP_OK) return fail(s);
  if (hflag) {
    set_last_error(hflag & BAD_PATTERN ? "gabp_create: the sparsity pattern is not symmetric"
                                       : "gabp_create: A_ij != A_ji");
    return fail(GABP_ERR_INVALID);
  }
  cudaFree(dflag);
  g.avg_deg = n > 0 ? (double)E / n : 0.0;
  return GABP_OK;
}

}  // namespace gabp

using namespace gabp;

extern "C" gabp_status gabp_options_default(gabp_options *o) {
  if (!o) return GABP_ERR_INVALID;
  memset(o, 0, sizeof(*o));
  o->variant = GABP_VARIANT_NODE;
  o->precision = GABP_PREC_FP64;
  o->check_every = 16;
  o->freeze_precisions = 0;
  o->inner_tol = 1e-4;
  o->inner_max_iter = 400;
  o->max_refine = 30;
  o->gamma_mode = 0;
  o->gamma = 0.25;
  o->lanes = 0;
  o->profile = 0;
  o->reuse_precisions = 1;
  o->multi_split = 0;
  o->prec_stop_log2 = 16;
  o->multi_mode = 0;
  o->overlap_precision = 1;
  o->device_loop = 1;
  o->fix_single_loop = 0;
  o->fix_step = 0.5;
  o->accel = 0;
  o->history = 0;
  o->warm_start = 0;
  o->initial_guess = 0;
  o->graphs = 1;
  o->reserved = 0;
  return GABP_OK;
}

static gabp_status check_options(const gabp_options *o) {
  if (o->variant != GABP_VARIANT_NODE && o->variant != GABP_VARIANT_EDGE) return GABP_ERR_INVALID;
  if (o->precision != GABP_PREC_FP64 && o->precision != GABP_PREC_FP32_REFINE) return GABP_ERR_INVALID;
  if (o->check_every < 1 || o->check_every > 4096) return GABP_ERR_INVALID;
  if (!(o->inner_tol > 0.0) || o->inner_max_iter < 1 || o->max_refine < 1) return GABP_ERR_INVALID;
  if (o->gamma_mode < 0 || o->gamma_mode > 2 || !(o->gamma >= 0.0)) return GABP_ERR_INVALID;
  if (o->lanes != 0 && (o->lanes < 1 || o->lanes > 32 || (o->lanes & (o->lanes - 1)))) return GABP_ERR_INVALID;
  if (o->unroll != 0 && o->unroll != 1 && o->unroll != 2 && o->unroll != 4 && o->unroll != 8) return GABP_ERR_INVALID;
  if (o->lanes && !pinned_shape32(o->lanes, o->unroll)) return GABP_ERR_INVALID;
  if ((o->profile != 0 && o->profile != 1) || (o->reuse_precisions != 0 && o->reuse_precisions != 1) ||
      o->multi_split < 0 || o->prec_stop_log2 < 10 || o->prec_stop_log2 > 23 || o->multi_mode < 0 ||
      o->multi_mode > 3 || o->overlap_precision < 0 || o->overlap_precision > 1 ||
      o->device_loop < 0 || o->device_loop > 1 || o->schedule < 0 || o->schedule > 1 || o->fix_single_loop < 0 ||
      o->fix_single_loop > 1 || !(o->fix_step > 0.0 && o->fix_step <= 1.0) || o->accel < 0 || o->accel > 2 || o->freeze_precisions < 0 || o->freeze_precisions > 1 || o->history < 0 || o->warm_start < 0 || o->warm_start > 1 || o->initial_guess < 0 || o->initial_guess > 1 || o->graphs < 0 || o->graphs > 1 ||
      (o->accel && o->variant != GABP_VARIANT_NODE) || (o->accel == 1 && o->schedule == 1))
    return GABP_ERR_INVALID;
  return GABP_OK;
}

namespace {
struct TunedShapes {
  int L64 = 0, Lp32 = 0, Lm32 = 0, Lj32 = 0;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int64_t>, TunedShapes> g_tune;
}  // namespace

void gabp::tune_cache_load(gabp_handle h) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(h->device, h->g.n, (int64_t)h->g.E));
  if (it == g_tune.end()) return;
  h->tuned_L64 = it->second.L64;
  h->tuned_Lp32 = it->second.Lp32;
  h->tuned_Lm32 = it->second.Lm32;
  h->tuned_Lj32 = it->second.Lj32;
}

void gabp::tune_cache_store(gabp_handle h) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  TunedShapes &t = g_tune[std::make_tuple(h->device, h->g.n, (int64_t)h->g.E)];
  if (h->tuned_L64) t.L64 = h->tuned_L64;
  if (h->tuned_Lp32) t.Lp32 = h->tuned_Lp32;
  if (h->tuned_Lm32) t.Lm32 = h->tuned_Lm32;
  if (h->tuned_Lj32) t.Lj32 = h->tuned_Lj32;
}

extern "C" gabp_status gabp_create(gabp_handle *out, int32_t n, int64_t nnz, const int32_t *rowptr,
                                   const int32_t *col, const double *val, int mem_space, void *stream,
                                   const gabp_options *opt) {
  if (!out) return GABP_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || nnz < n || nnz >= INT32_MAX || !rowptr || !col || !val || (mem_space != 0 && mem_space != 1)) {
    set_last_error("gabp_create: invalid argument");
    return GABP_ERR_INVALID;
  }
  gabp_options o;
  gabp_options_default(&o);
  if (opt) o = *opt;
  if (check_options(&o) != GABP_OK) {
    set_last_error("gabp_create: invalid options");
    return GABP_ERR_INVALID;
  }
  gabp_handle h = new (std::nothrow) gabp_handle_s();
  if (!h) return GABP_ERR_NOMEM;
  h->opt = o;
  h->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess && !h->stream) {  // no stream given: a stream of the handle's own (see order_after_caller)
    e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->caller_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
      h->stream = h->own_stream;
      h->order_legacy = true;
    }
  }
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    gabp_status s = cuda_fail(e, "gabp_create device query");
    delete h;
    return s;
  }
  h->max_blocks = h->num_sms * 8;
  gabp_status s = GABP_OK;
  if ((e = cudaEventCreate(&h->prof.e0)) != cudaSuccess || (e = cudaEventCreate(&h->prof.e1)) != cudaSuccess ||
      (e = cudaMalloc(&h->ctl, sizeof(DevCtl))) != cudaSuccess ||
      (e = cudaMallocHost(&h->ctl_host, sizeof(DevCtl))) != cudaSuccess ||
      (e = cudaMalloc(&h->partials, sizeof(double) * 4 * h->max_blocks)) != cudaSuccess) {
    s = cuda_fail(e, "gabp_create control block");
  }
  if (s == GABP_OK) s = create_impl(h, n, nnz, rowptr, col, val, mem_space);
  if (s == GABP_OK) {
    e = cudaMemsetAsync(h->ctl, 0, sizeof(DevCtl), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) s = cuda_fail(e, "gabp_create finish");
  }
  if (s != GABP_OK) {
    destroy_impl(h);
    return s;
  }
  tune_cache_load(h);
  *out = h;
  return GABP_OK;
}

extern "C" gabp_status gabp_set_values(gabp_handle h, const double *val, int mem_space) {
  if (!h || !val || (mem_space != 0 && mem_space != 1)) return GABP_ERR_INVALID;
  DeviceGuard dg(h->device);
  order_after_caller(h);
  Graph &g = h->g;
  h->values_ok = false;  // until the new values pass every check
  h->last_path = -1;     // marginals / messages of the old values are gone
  h->w64.valid = false;  // and no warm start from them
  h->w64.sl.vals_ok = false;  // the sliced copy of the values is refreshed by the next FP64 solve
  if (h->gsl) h->gsl->vals_ok = false;  // and the independent-systems one by the next such solve
  h->w32.coef_ready = false;
  h->w32.prec_round = -1;
  int *dflag = nullptr;
  GABP_CUDA(cudaMalloc(&dflag, sizeof(int)));
  struct F {
    int *p;
    ~F() { cudaFree(p); }
  } fr{dflag};
  int hflag = 0;
  auto read_flag = [&]() -> gabp_status {
    cudaError_t e = cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "validation read-back");
    return GABP_OK;
  };
  GABP_CUDA(cudaMemcpyAsync(g.val, val, sizeof(double) * g.nnz,
                            mem_space == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream));
  GABP_CUDA(cudaMemsetAsync(dflag, 0, sizeof(int), h->stream));
  const int nb = (g.n + kBlock - 1) / kBlock;
  k_check_rows<<<nb, kBlock, 0, h->stream>>>(g.n, g.rowptr, g.col, g.val, g.dpos, dflag);
  gabp_status s = read_flag();
  if (s != GABP_OK) return s;
  if (hflag) {
    set_last_error(hflag & BAD_DIAG ? "gabp_set_values: a diagonal entry is zero or non-finite"
                                    : "gabp_set_values: zero or non-finite off-diagonal entry");
    return GABP_ERR_INVALID;
  }
  k_compact<<<(g.n + 1 + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, g.rowptr, g.col, g.val, g.dpos, g.rp,
                                                                        g.ci, g.av, g.ad);
  if (g.E > 0)
    k_check_sym<<<(int)(((int64_t)g.E + kBlock - 1) / kBlock), kBlock, 0, h->stream>>>(g.E, g.av, g.rev, dflag);
  if ((s = read_flag()) != GABP_OK) return s;
  if (hflag) {
    set_last_error("gabp_set_values: A_ij != A_ji");
    return GABP_ERR_INVALID;
  }
  if (g.av32 && g.E > 0) {
    k_values_to_f32<<<(int)(((int64_t)g.E + kBlock - 1) / kBlock), kBlock, 0, h->stream>>>(g.E, g.av, g.av32);
    GABP_CUDA(cudaGetLastError());
  }
  if ((s = serial_refresh_values(h)) != GABP_OK) return s;
  h->values_ok = true;
  return GABP_OK;
}

extern "C" gabp_status gabp_set_options(gabp_handle h, const gabp_options *opt) {
  if (!h || !opt || check_options(opt) != GABP_OK) return GABP_ERR_INVALID;
  bool rebuild = opt->variant != h->opt.variant || opt->lanes != h->opt.lanes || opt->unroll != h->opt.unroll ||
                 opt->check_every != h->opt.check_every ||
                 opt->accel != h->opt.accel;
  h->opt = *opt;
  if (rebuild) {
    if (h->g64) cudaGraphExecDestroy(h->g64);
    h->g64 = nullptr;
    h->g64_key = -1;
    if (h->gP32) cudaGraphExecDestroy(h->gP32);
    h->gP32 = nullptr;
    if (h->gH32) cudaGraphExecDestroy(h->gH32);
    h->gH32 = nullptr;
    if (h->gJ32) cudaGraphExecDestroy(h->gJ32);
    h->gJ32 = nullptr;
    if (h->gRef) cudaGraphExecDestroy(h->gRef);
    if (h->gRefG) cudaGraphDestroy(h->gRefG);
    h->gRef = nullptr;
    h->gRefG = nullptr;
    h->gRef_key = -1;
    h->gH32_R = -1;
  }
  return GABP_OK;
}

extern "C" gabp_status gabp_set_stream(gabp_handle h, void *stream) {
  if (!h) return GABP_ERR_INVALID;
  DeviceGuard dg(h->device);
  if (h->stream) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "gabp_set_stream");
  }
  if (stream) {
    h->stream = (cudaStream_t)stream;
    h->order_legacy = false;
  } else {  // back to the handle's own stream, ordered after the legacy default stream
    if (!h->own_stream) {
      cudaError_t e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess && !h->caller_ev) e = cudaEventCreateWithFlags(&h->caller_ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(e, "gabp_set_stream");
    }
    h->stream = h->own_stream;
    h->order_legacy = true;
  }
  return GABP_OK;
}

extern "C" gabp_status gabp_destroy(gabp_handle h) { return destroy_impl(h); }

extern "C" const char *gabp_status_string(gabp_status s) {
  switch (s) {
    case GABP_OK: return "converged";
    case GABP_NOT_CONVERGED: return "not converged within max_iter";
    case GABP_DIVERGED: return "diverged (non-finite value)";
    case GABP_BREAKDOWN: return "breakdown (zero cavity or marginal precision)";
    case GABP_TIMEOUT: return "device-side wait timed out";
    case GABP_ERR_INVALID: return "invalid argument or matrix";
    case GABP_ERR_CUDA: return "CUDA error";
    case GABP_ERR_NOMEM: return "out of device memory";
  }
  return "unknown status";
}

extern "C" const char *gabp_last_error(void) { return g_last_error.c_str(); }
