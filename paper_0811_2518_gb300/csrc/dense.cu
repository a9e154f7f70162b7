// dense.cu -- gabp_create_dense: a handle for a dense symmetric matrix.
//
// The broadcast form of GaBP (Algorithm 2) needs nothing of A's sparsity: every
// node forms its aggregates P~_i, h~_i and each incoming message comes from the
// sender's aggregate minus the reverse message.  On a dense matrix -- the kernel
// matrices of the regression chapter (support vector and kernel ridge regression,
// where the paper broadcasts the n aggregates every round) -- a row's slots are
// all the other columns, so the round kernels' per-slot gathers of the senders'
// aggregates become sequential reads of one n-vector.  The entry builds the
// row-CSR of A's nonzero entries (the diagonal always kept) on the device and
// creates an ordinary handle on it: every solve path, the refinement, the
// precision freeze and the batched solves apply unchanged.
#include "gabp_internal.cuh"

#include <vector>

namespace gabp {
namespace {

// entries kept in row i: nonzeros and the diagonal (NaN counts as nonzero, and is
// then rejected by the matrix validation)
__device__ __forceinline__ bool kept(double v, int i, int j) { return v != 0.0 || i == j; }

// a warp per row: number of kept entries
__global__ void k_dense_count(int n, const double *__restrict__ A, int64_t lda, int *cnt) {
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const double *row = A + (size_t)i * lda;
  int c = 0;
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + lane;
    const bool k = j < n && kept(row[j], i, j);
    c += __popc(__ballot_sync(0xffffffffu, k));
  }
  if (lane == 0) cnt[i] = c;
}

// a warp per row: the kept entries in column order at rowptr[i]..
__global__ void k_dense_fill(int n, const double *__restrict__ A, int64_t lda, const int *__restrict__ rowptr,
                             int *col, double *val) {
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const double *row = A + (size_t)i * lda;
  int base = rowptr[i];
  const unsigned below = (1u << lane) - 1u;
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + lane;
    const double v = j < n ? row[j] : 0.0;
    const bool k = j < n && kept(v, i, j);
    const unsigned m = __ballot_sync(0xffffffffu, k);
    if (k) {
      const int p = base + __popc(m & below);
      col[p] = j;
      val[p] = v;
    }
    base += __popc(m);
  }
}

}  // namespace
}  // namespace gabp

using namespace gabp;

extern "C" gabp_status gabp_create_dense(gabp_handle *out, int32_t n, const double *A, int64_t lda, int mem_space,
                                        void *stream, const gabp_options *opt, int64_t *nnz_out) {
  if (!out) return GABP_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || !A || lda < n || (mem_space != 0 && mem_space != 1)) {
    set_last_error("gabp_create_dense: invalid argument");
    return GABP_ERR_INVALID;
  }
  if (mem_space == 1 && !is_device_ptr(A)) {
    set_last_error("gabp_create_dense: mem_space = 1 needs a device array");
    return GABP_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  struct Free {
    std::vector<void *> p;
    ~Free() { for (void *q : p) cudaFree(q); }
  } fr;
  const double *dA = A;
  int64_t dlda = lda;
  if (mem_space == 0) {  // the host matrix to the device, rows packed
    double *t = nullptr;
    GABP_CUDA(cudaMalloc(&t, sizeof(double) * (size_t)n * n));
    fr.p.push_back(t);
    GABP_CUDA(cudaMemcpy2DAsync(t, sizeof(double) * n, A, sizeof(double) * lda, sizeof(double) * n, n,
                                cudaMemcpyHostToDevice, st));
    dA = t;
    dlda = n;
  }
  int *cnt = nullptr;
  GABP_CUDA(cudaMalloc(&cnt, sizeof(int) * (size_t)(n + 1)));
  fr.p.push_back(cnt);
  const int warps_per_block = kBlock / 32;
  const int nb = (n + warps_per_block - 1) / warps_per_block;
  k_dense_count<<<nb, kBlock, 0, st>>>(n, dA, dlda, cnt);
  GABP_CUDA(cudaGetLastError());
  std::vector<int> c(n);
  GABP_CUDA(cudaMemcpyAsync(c.data(), cnt, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  GABP_CUDA(cudaStreamSynchronize(st));
  std::vector<int> rp(n + 1, 0);
  int64_t nnz = 0;
  for (int i = 0; i < n; ++i) {
    nnz += c[i];
    if (nnz >= INT32_MAX) {
      set_last_error("gabp_create_dense: more than 2^31 - 1 kept entries");
      return GABP_ERR_INVALID;
    }
    rp[i + 1] = (int)nnz;
  }
  int *drp = nullptr, *dcol = nullptr;
  double *dval = nullptr;
  GABP_CUDA(cudaMalloc(&drp, sizeof(int) * (size_t)(n + 1)));
  fr.p.push_back(drp);
  GABP_CUDA(cudaMalloc(&dcol, sizeof(int) * (size_t)nnz));
  fr.p.push_back(dcol);
  GABP_CUDA(cudaMalloc(&dval, sizeof(double) * (size_t)nnz));
  fr.p.push_back(dval);
  GABP_CUDA(cudaMemcpyAsync(drp, rp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
  k_dense_fill<<<nb, kBlock, 0, st>>>(n, dA, dlda, drp, dcol, dval);
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(st));  // the CSR is complete before the handle reads it
  if (nnz_out) *nnz_out = nnz;
  return gabp_create(out, n, nnz, drp, dcol, dval, 1, stream, opt);
}
