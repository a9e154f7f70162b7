// noalloc.cu -- gabp_solve_noalloc: an FP64 GaBP solve that allocates nothing.
//
// Why it exists.  gabp_create / gabp_solve take their working memory (messages,
// node records, the reverse-edge index) from cudaMalloc.  Some callers cannot
// do that at solve time: a latency-critical loop cannot afford cudaMalloc's
// device-wide synchronisation and unbounded latency; a process whose device
// memory has been reserved up front by another allocator may see cudaMalloc
// fail; and code written under rules that forbid dynamic allocation after
// start-up may not call it at all.  This entry point takes its scratch from
// one fixed array in the library's own device memory instead.
//
// The scratch is a file-scope __device__ array of kScratchBytes (about 5.6 MB).
// Every GPU that loads the library holds it until the process exits.  It bounds
// the problem size: n <= 16384 and nnz <= 131072 (full CSR, diagonal included);
// larger inputs are rejected with GABP_ERR_INVALID before anything is launched.
//
// Host code may not use the array's name as a device address (in host code it
// names a host-side stand-in).  The first call on each device therefore looks
// the address up with cudaGetSymbolAddress, with that device current, checks
// the result and caches it for the life of the process; later calls reuse the
// cached address.  A cudaDeviceReset invalidates that address: calls after a
// reset of the device are not supported.
//
// Every call ends by copying the run's status to the host and synchronising the
// caller's stream, so the function cannot be called while that stream is being
// captured into a CUDA graph.  The five arrays must be device (or managed)
// memory: host pointers are rejected before anything is launched.
//
// All calls share the one array and it keeps whatever the last call left in
// it: the kernel clears what must start at zero (the round-0 messages) and
// rebuilds everything else before use.  Calls that overlap on the GPU (two
// streams, two host threads, or two devices' work aimed at the same device's
// array) race on the scratch and give wrong answers; serialise them.
//
// The computation is the plain FP64 path of gabp_solve (Algorithm 2 of the
// paper, synchronous schedule, information-form messages), run by one thread
// block for all rounds of the solve.
#include "gabp_internal.cuh"
#include "devutil.cuh"

#include <mutex>

namespace {

using gabp::kBlock;
using gabp::NodeRec64;

constexpr int kNaMaxN = 16384;
constexpr int kNaMaxNnz = 131072;
constexpr int kNaMaxDevices = 64;

constexpr size_t round256(size_t v) { return (v + 255) / 256 * 256; }

struct NaCtl {
  int status;
  int iters;
  double relres;
};

constexpr size_t kOffCtl = 0;
constexpr size_t kOffRev = 256;
constexpr size_t kOffM0 = kOffRev + round256(sizeof(int) * kNaMaxNnz);
constexpr size_t kOffM1 = kOffM0 + round256(sizeof(double2) * kNaMaxNnz);
constexpr size_t kOffN0 = kOffM1 + round256(sizeof(double2) * kNaMaxNnz);
constexpr size_t kOffN1 = kOffN0 + round256(sizeof(NodeRec64) * kNaMaxN);
constexpr size_t kScratchBytes = kOffN1 + round256(sizeof(NodeRec64) * kNaMaxN);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// One block does everything: input checks, the reverse-edge index, round 0,
// then rounds t = 1..max_iter until ||b - A x_t|| <= tol ||b|| (Algorithm 1
// step 3 with the residual rule), a zero cavity / marginal precision
// (breakdown) or a non-finite residual (divergence).
__global__ void __launch_bounds__(kBlock) k_noalloc_solve(int n, int nnz, const int *__restrict__ rowptr,
                                                          const int *__restrict__ col,
                                                          const double *__restrict__ val,
                                                          const double *__restrict__ b, double *__restrict__ x,
                                                          double tol, int max_iter, unsigned char *scratch) {
  NaCtl *ctl = reinterpret_cast<NaCtl *>(scratch + kOffCtl);
  int *rev = reinterpret_cast<int *>(scratch + kOffRev);
  double2 *M0 = reinterpret_cast<double2 *>(scratch + kOffM0);
  double2 *M1 = reinterpret_cast<double2 *>(scratch + kOffM1);
  NodeRec64 *N0 = reinterpret_cast<NodeRec64 *>(scratch + kOffN0);
  NodeRec64 *N1 = reinterpret_cast<NodeRec64 *>(scratch + kOffN1);
  __shared__ int s_flag;
  __shared__ int s_done, s_result;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) s_flag = 0;
  __syncthreads();

  // checks 1: rowptr is a valid CSR row pointer
  for (int i = tid; i < n; i += nt) {
    int a = rowptr[i], c = rowptr[i + 1];
    if (a > c || a < 0 || c > nnz || (i == 0 && a != 0) || (i == n - 1 && c != nnz)) atomicOr(&s_flag, 1);
  }
  __syncthreads();
  if (s_flag) {
    if (tid == 0) { ctl->status = GABP_ERR_INVALID; ctl->iters = 0; ctl->relres = 0.0; }
    return;
  }
  // checks 2: sorted in-range columns, one nonzero finite diagonal, nonzero finite off-diagonals
  for (int i = tid; i < n; i += nt) {
    int nd = 0, prev = -1;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      int c = col[p];
      double v = val[p];
      if (c < 0 || c >= n || c <= prev || v == 0.0 || !isfinite(v)) atomicOr(&s_flag, 2);
      prev = c;
      nd += (c == i);
    }
    if (nd != 1) atomicOr(&s_flag, 2);
  }
  __syncthreads();
  if (s_flag) {
    if (tid == 0) { ctl->status = GABP_ERR_INVALID; ctl->iters = 0; ctl->relres = 0.0; }
    return;
  }
  // checks 3 + set-up: reverse slots (symmetric pattern and values), round-0 state
  double bb = 0.0;
  for (int i = tid; i < n; i += nt) {
    double d = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      int k = col[p];
      M0[p] = make_double2(0.0, 0.0);  // round-0 messages are zero (Algorithm 1, step 1)
      if (k == i) { d = val[p]; rev[p] = p; continue; }
      int lo = rowptr[k], hi = rowptr[k + 1] - 1, hit = -1;
      while (lo <= hi) {
        int mid = (lo + hi) >> 1, c = col[mid];
        if (c == i) { hit = mid; break; }
        if (c < i) lo = mid + 1; else hi = mid - 1;
      }
      if (hit < 0 || __double_as_longlong(val[hit]) != __double_as_longlong(val[p])) {
        atomicOr(&s_flag, 4);
        rev[p] = p;
      } else {
        rev[p] = hit;
      }
    }
    double bi = b[i];
    N0[i] = NodeRec64{d, bi, bi / d, 0.0};
    bb = fma(bi, bi, bb);
  }
  double vb[1] = {bb};
  gabp::block_sum<1>(vb);  // block_sum ends with a barrier
  __shared__ double s_bb;
  if (tid == 0) s_bb = vb[0];
  __syncthreads();
  if (s_flag) {
    if (tid == 0) { ctl->status = GABP_ERR_INVALID; ctl->iters = 0; ctl->relres = 0.0; }
    return;
  }
  bb = s_bb;
  if (bb == 0.0) {
    for (int i = tid; i < n; i += nt) x[i] = 0.0;
    if (tid == 0) { ctl->status = GABP_OK; ctl->iters = 0; ctl->relres = 0.0; }
    return;
  }
  {  // residual of the round-0 iterate x_0 = b_i / A_ii (reported if max_iter = 0)
    double rr = 0.0;
    for (int i = tid; i < n; i += nt) {
      double ax = 0.0;
      for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) ax = fma(val[p], N0[col[p]].x, ax);
      const double r = b[i] - ax;
      rr = fma(r, r, rr);
    }
    double v[1] = {rr};
    gabp::block_sum<1>(v);
    if (tid == 0) { s_done = 0; s_result = 0; ctl->status = GABP_NOT_CONVERGED; ctl->iters = 0; ctl->relres = sqrt(v[0] / bb); }
    __syncthreads();
  }
  const double tol2bb = tol * tol * bb;
  for (int t = 1; t <= max_iter; ++t) {
    const double2 *Min = (t & 1) ? M0 : M1;
    double2 *Mout = (t & 1) ? M1 : M0;
    const NodeRec64 *Nin = (t & 1) ? N0 : N1;
    NodeRec64 *Nout = (t & 1) ? N1 : N0;
    double bad = 0.0;
    for (int i = tid; i < n; i += nt) {
      double accP = 0.0, acch = 0.0, d = 0.0;
      for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        const int k = col[p];
        if (k == i) { d = val[p]; continue; }
        const double A = val[p];
        const double2 rv = Min[rev[p]];   // message i -> k of round t-1
        const NodeRec64 nk = Nin[k];      // node k at round t-1
        const double den = nk.P - rv.x;   // cavity precision of k without i
        if (den == 0.0) bad += 1.0;
        const double cin = -A * gabp::rcp64(den);
        const double2 m = make_double2(cin * A, cin * (nk.h - rv.y));
        Mout[p] = m;
        accP += m.x;
        acch += m.y;
      }
      const double P = d + accP, h = b[i] + acch;
      if (P == 0.0) bad += 1.0;
      Nout[i] = NodeRec64{P, h, h / P, 0.0};
    }
    __syncthreads();
    double rr = 0.0;
    for (int i = tid; i < n; i += nt) {
      double ax = 0.0;
      for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) ax = fma(val[p], Nout[col[p]].x, ax);
      const double r = b[i] - ax;
      rr = fma(r, r, rr);
    }
    double v[2] = {rr, bad};
    gabp::block_sum<2>(v);
    if (tid == 0) {
      if (v[1] > 0.0) {
        ctl->status = GABP_BREAKDOWN; ctl->iters = t; s_result = t - 1; s_done = 1;
      } else if (!isfinite(v[0])) {
        ctl->status = GABP_DIVERGED; ctl->iters = t; ctl->relres = sqrt(v[0] / bb); s_result = t; s_done = 1;
      } else {
        ctl->relres = sqrt(v[0] / bb);
        ctl->iters = t;
        s_result = t;
        if (v[0] <= tol2bb) { ctl->status = GABP_OK; s_done = 1; }
      }
    }
    __syncthreads();
    if (s_done) break;
  }
  const NodeRec64 *Nr = (s_result & 1) ? N1 : N0;
  for (int i = tid; i < n; i += nt) x[i] = Nr[i].x;
}

std::mutex g_mu;
void *g_addr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
gabp_status scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gabp::cuda_fail(e, "gabp_solve_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kNaMaxDevices) {
    gabp::set_last_error("gabp_solve_noalloc: device ordinal out of range");
    return GABP_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return gabp::cuda_fail(e, "gabp_solve_noalloc: cudaGetSymbolAddress");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return GABP_OK;
}

}  // namespace

extern "C" gabp_status gabp_solve_noalloc(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                                          const double *val, const double *b, double *x, double tol,
                                          int32_t max_iter, void *stream, int32_t *iters_out,
                                          double *relres_out) {
  if (n < 1 || n > kNaMaxN || nnz < n || nnz > kNaMaxNnz) {
    gabp::set_last_error("gabp_solve_noalloc: size out of range (needs 1 <= n <= 16384 and n <= nnz <= 131072)");
    return GABP_ERR_INVALID;
  }
  if (!rowptr || !col || !val || !b || !x || !(tol >= 0.0) || max_iter < 0) {
    gabp::set_last_error("gabp_solve_noalloc: invalid argument");
    return GABP_ERR_INVALID;
  }
  // the kernel dereferences all five: a host address would fault on the device
  if (!gabp::is_device_ptr(rowptr) || !gabp::is_device_ptr(col) || !gabp::is_device_ptr(val) ||
      !gabp::is_device_ptr(b) || !gabp::is_device_ptr(x)) {
    gabp::set_last_error("gabp_solve_noalloc: rowptr, col, val, b and x must be device arrays");
    return GABP_ERR_INVALID;
  }
  void *scratch = nullptr;
  gabp_status s = scratch_address(&scratch);
  if (s != GABP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  k_noalloc_solve<<<1, kBlock, 0, st>>>(n, (int)nnz, rowptr, col, val, b, x, tol, max_iter,
                                        static_cast<unsigned char *>(scratch));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gabp::cuda_fail(e, "gabp_solve_noalloc: launch");
  NaCtl c;
  e = cudaMemcpyAsync(&c, static_cast<unsigned char *>(scratch) + kOffCtl, sizeof(c), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return gabp::cuda_fail(e, "gabp_solve_noalloc: read-back");
  if (c.status == GABP_ERR_INVALID) {
    gabp::set_last_error("gabp_solve_noalloc: matrix rejected (CSR structure, diagonal or symmetry)");
    return GABP_ERR_INVALID;
  }
  if (iters_out) *iters_out = c.iters;
  if (relres_out) *relres_out = c.relres;
  return (gabp_status)c.status;
}
