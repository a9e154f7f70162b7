// lsq.cu -- regularised least squares / MMSE solutions of a rectangular system by GaBP.
//
// Paper: Sec. "Extension to General Linear Systems" and Chapter "Extending GaBP to
// support non-square matrices".  For a rectangular J (m x k) and y (m), the symmetric
// augmented system
//     [ I_k   J^T      ] [x]   [0]
//     [ J    -gamma I_m] [z] = [y]
// has x = (J^T J + gamma I)^{-1} J^T y (second block row: z = (J x - y) / gamma; first:
// x = -J^T z), the regularised least-squares solution, and the MMSE detector of the
// non-square chapter with Psi = gamma I.  It is sparse (2 nnz(J) off-diagonal entries,
// no J^T J is formed), so every solver path of the library runs on it unchanged.
//
// gabp_create_lsq assembles the augmented full symmetric CSR (variables x first,
// auxiliary z after them) in host memory -- a one-time O(nnz) counting-sort transpose
// of J -- and creates an ordinary handle on it; gabp_solve_lsq stages [0; y], runs the
// handle's solve path and splits the marginal means into x and z.
#include "gabp_internal.cuh"

#include <cmath>
#include <vector>

using namespace gabp;

extern "C" gabp_status gabp_create_lsq(gabp_handle *out, int32_t m, int32_t k, int64_t nnz, const int32_t *rowptr,
                                       const int32_t *col, const double *val, double gamma, int mem_space,
                                       void *stream, const gabp_options *opt) {
  if (!out) return GABP_ERR_INVALID;
  *out = nullptr;
  if (m < 1 || k < 1 || nnz < 0 || !rowptr || (nnz > 0 && (!col || !val)) || (mem_space != 0 && mem_space != 1) ||
      !(gamma > 0.0) || !std::isfinite(gamma)) {
    set_last_error("gabp_create_lsq: invalid argument");
    return GABP_ERR_INVALID;
  }
  const int64_t n = (int64_t)k + m, nnz_aug = n + 2 * nnz;
  if (n >= INT32_MAX || nnz_aug >= INT32_MAX) {
    set_last_error("gabp_create_lsq: the augmented system does not fit int32 indices");
    return GABP_ERR_INVALID;
  }
  // J in host memory
  std::vector<int32_t> rp((size_t)m + 1), ci((size_t)nnz);
  std::vector<double> v((size_t)nnz);
  if (mem_space == 1) {
    if (stream) GABP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    GABP_CUDA(cudaMemcpy(rp.data(), rowptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost));
    if (nnz > 0) {
      GABP_CUDA(cudaMemcpy(ci.data(), col, sizeof(int32_t) * ci.size(), cudaMemcpyDeviceToHost));
      GABP_CUDA(cudaMemcpy(v.data(), val, sizeof(double) * v.size(), cudaMemcpyDeviceToHost));
    }
  } else {
    std::copy(rowptr, rowptr + m + 1, rp.begin());
    if (nnz > 0) {
      std::copy(col, col + nnz, ci.begin());
      std::copy(val, val + nnz, v.begin());
    }
  }
  // validation: a CSR row pointer from 0 to nnz, strictly increasing columns in [0, k),
  // finite nonzero values (a stored zero would be an edge that carries nothing)
  if (rp[0] != 0 || rp[m] != nnz) {
    set_last_error("gabp_create_lsq: rowptr must run from 0 to nnz");
    return GABP_ERR_INVALID;
  }
  for (int32_t r = 0; r < m; ++r) {
    if (rp[r + 1] < rp[r]) {
      set_last_error("gabp_create_lsq: rowptr is not monotone");
      return GABP_ERR_INVALID;
    }
    for (int64_t p = rp[r]; p < rp[r + 1]; ++p) {
      if (ci[p] < 0 || ci[p] >= k || (p > rp[r] && ci[p] <= ci[p - 1])) {
        set_last_error("gabp_create_lsq: column index out of range or not strictly increasing");
        return GABP_ERR_INVALID;
      }
      if (!(v[p] != 0.0) || !std::isfinite(v[p])) {
        set_last_error("gabp_create_lsq: zero or non-finite entry of J");
        return GABP_ERR_INVALID;
      }
    }
  }
  // J^T by a counting sort over the columns; rows stay ascending within a column
  std::vector<int64_t> cp((size_t)k + 1, 0);
  for (int64_t p = 0; p < nnz; ++p) ++cp[(size_t)ci[p] + 1];
  for (int32_t c = 0; c < k; ++c) cp[c + 1] += cp[c];
  std::vector<int32_t> tr((size_t)nnz);
  std::vector<double> tv((size_t)nnz);
  {
    std::vector<int64_t> fill(cp.begin(), cp.end() - 1);
    for (int32_t r = 0; r < m; ++r)
      for (int64_t p = rp[r]; p < rp[r + 1]; ++p) {
        const int64_t q = fill[ci[p]]++;
        tr[q] = r;
        tv[q] = v[p];
      }
  }
  // the augmented full symmetric CSR: row c < k is (c: 1, k + r: J_rc for r ascending);
  // row k + r is (c: J_rc for c ascending, k + r: -gamma)
  std::vector<int32_t> arp((size_t)n + 1), aci((size_t)nnz_aug);
  std::vector<double> av((size_t)nnz_aug);
  int64_t w = 0;
  for (int32_t c = 0; c < k; ++c) {
    arp[c] = (int32_t)w;
    aci[w] = c;
    av[w++] = 1.0;
    for (int64_t q = cp[c]; q < cp[c + 1]; ++q) {
      aci[w] = k + tr[q];
      av[w++] = tv[q];
    }
  }
  for (int32_t r = 0; r < m; ++r) {
    arp[(size_t)k + r] = (int32_t)w;
    for (int64_t p = rp[r]; p < rp[r + 1]; ++p) {
      aci[w] = ci[p];
      av[w++] = v[p];
    }
    aci[w] = k + r;
    av[w++] = -gamma;
  }
  arp[n] = (int32_t)w;
  gabp_handle h = nullptr;
  gabp_status s = gabp_create(&h, (int32_t)n, nnz_aug, arp.data(), aci.data(), av.data(), 0, stream, opt);
  if (s != GABP_OK) return s;
  h->lsq_m = m;
  h->lsq_k = k;
  *out = h;
  return GABP_OK;
}

extern "C" gabp_status gabp_solve_lsq(gabp_handle h, const double *y, double *x, double *z, double tol,
                                      int32_t max_iter, int32_t *iters_out, double *relres_out) {
  if (!h || !y || !x || h->lsq_k < 1) {
    set_last_error("gabp_solve_lsq: invalid argument or not a least-squares handle");
    return GABP_ERR_INVALID;
  }
  if (h->opt.initial_guess) {
    set_last_error("gabp_solve_lsq: options.initial_guess is not supported");
    return GABP_ERR_INVALID;
  }
  if (!is_device_ptr(y) || !is_device_ptr(x) || (z && !is_device_ptr(z))) {
    set_last_error("gabp_solve_lsq: y, x and z must be device arrays");
    return GABP_ERR_INVALID;
  }
  DeviceGuard dg(h->device);
  order_after_caller(h);
  const size_t n = (size_t)h->g.n, k = (size_t)h->lsq_k, m = (size_t)h->lsq_m;
  if (!h->lsq_b) GABP_CUDA(cudaMalloc(&h->lsq_b, sizeof(double) * n));
  if (!h->lsq_x) GABP_CUDA(cudaMalloc(&h->lsq_x, sizeof(double) * n));
  GABP_CUDA(cudaMemsetAsync(h->lsq_b, 0, sizeof(double) * k, h->stream));
  GABP_CUDA(cudaMemcpyAsync(h->lsq_b + k, y, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->stream));
  gabp_status s = solve_dispatch(h, h->lsq_b, h->lsq_x, tol, max_iter, iters_out, relres_out);
  if (s < 0) return s;
  GABP_CUDA(cudaMemcpyAsync(x, h->lsq_x, sizeof(double) * k, cudaMemcpyDeviceToDevice, h->stream));
  if (z) GABP_CUDA(cudaMemcpyAsync(z, h->lsq_x + k, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return s;
}
