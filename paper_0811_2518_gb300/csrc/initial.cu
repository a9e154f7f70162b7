// initial.cu -- solves that start from a caller's iterate x0 (options.initial_guess).
//
// Every path solves A x = b from x = 0.  With an initial iterate the same path
// solves the correction system A d = r0, r0 = b - A x0 (FP64), and returns
// x = x0 + d.  The stop rule of the original system, ||b - A x|| <= tol ||b||,
// is ||r0 - A d|| <= tol ||b||, i.e. the correction solve runs with the
// tolerance tol ||b|| / ||r0||.  A good x0 leaves a small r0, so the solve needs
// fewer rounds (a sequence of nearby right-hand sides, a restarted solve).
#include "gabp_internal.cuh"
#include "devutil.cuh"

#include <cmath>

namespace gabp {

namespace {

// r0 = b - A x0 over the full CSR (FP64) with the sums ||r0||^2 and ||b||^2.
template <int L>
__global__ void __launch_bounds__(kBlock) k_ig_residual(int n, const int *__restrict__ rowptr,
                                                        const int *__restrict__ col, const double *__restrict__ val,
                                                        const double *__restrict__ b, const double *__restrict__ x0,
                                                        double *__restrict__ r0, double *sums, double *partials,
                                                        unsigned int *arrive) {
  constexpr int RPW = 32 / L;
  const int lane = threadIdx.x & 31, sl = lane & (L - 1), sw = lane / L;
  const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  double rr = 0.0, bb = 0.0;
  for (int base = warp * RPW; base < n; base += nwarps * RPW) {
    const int i = base + sw;
    double ax = 0.0;
    if (i < n)
      for (int p = rowptr[i] + sl; p < rowptr[i + 1]; p += L) ax = fma(val[p], x0[col[p]], ax);
    ax = sub_sum<L>(ax);
    if (i < n && sl == 0) {
      const double bi = b[i], r = bi - ax;
      r0[i] = r;
      rr = fma(r, r, rr);
      bb = fma(bi, bi, bb);
    }
  }
  double v[2] = {rr, bb}, tot[2];
  const int modes[2] = {0, 0};
  block_sum<2>(v);
  if (last_block_reduce<2>(v, modes, partials, arrive, tot) && threadIdx.x == 0) {
    sums[0] = tot[0];
    sums[1] = tot[1];
    *arrive = 0;
    __threadfence();
  }
}

__global__ void k_ig_add(int n, double *__restrict__ x, const double *__restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += d[i];
}

}  // namespace

// x holds x0 on entry and the answer on return; solve(r0, d, tol') runs the path.
gabp_status solve_from_initial(gabp_handle h, const double *b, double *x, double tol, int *iters, double *relres,
                               const std::function<gabp_status(const double *, double *, double, int *, double *)>
                                   &solve) {
  Graph &g = h->g;
  const size_t n = (size_t)g.n;
  if (!h->ig_buf) {
    GABP_CUDA(cudaMalloc(&h->ig_buf, sizeof(double) * (2 * n + 2) + sizeof(unsigned int) * 4));
    GABP_CUDA(cudaMemsetAsync(h->ig_buf, 0, sizeof(double) * (2 * n + 2) + sizeof(unsigned int) * 4, h->stream));
  }
  double *r0 = h->ig_buf, *d = h->ig_buf + n, *sums = h->ig_buf + 2 * n;
  unsigned int *arrive = reinterpret_cast<unsigned int *>(sums + 2);
  const int L = g.avg_deg >= 12.0 ? 2 : 1;
  GABP_DISPATCH_L(L, {
    const int nb = blocks_for(g.n, kBlock / LL, resident_grid(h->num_sms, k_ig_residual<LL>));
    (k_ig_residual<LL><<<nb, kBlock, 0, h->stream>>>(g.n, g.rowptr, g.col, g.val, b, x, r0, sums, h->partials,
                                                     arrive));
  });
  GABP_CUDA(cudaGetLastError());
  double hs[2] = {0.0, 0.0};
  GABP_CUDA(cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  const double rr0 = hs[0], bb = hs[1];
  if (!std::isfinite(rr0)) {
    set_last_error("initial guess: the residual b - A x0 is not finite");
    return GABP_ERR_INVALID;
  }
  if (bb == 0.0) {  // b = 0: x = 0, whatever x0 was
    GABP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, h->stream));
    GABP_CUDA(cudaStreamSynchronize(h->stream));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return GABP_OK;
  }
  if (rr0 <= tol * tol * bb) {  // x0 already meets the tolerance
    if (iters) *iters = 0;
    if (relres) *relres = std::sqrt(rr0 / bb);
    return GABP_OK;
  }
  const double scale = std::sqrt(bb / rr0);  // ||b|| / ||r0||
  int it = 0;
  double rel = 0.0;
  const gabp_status s = solve(r0, d, tol * scale, &it, &rel);
  if (s < 0) return s;
  h->hist_bb = bb;  // a recorded history holds ||r0 - A d_t|| = ||b - A (x0 + d_t)||: relative to ||b||
  k_ig_add<<<(g.n + kBlock - 1) / kBlock, kBlock, 0, h->stream>>>(g.n, x, d);
  GABP_CUDA(cudaGetLastError());
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  if (iters) *iters = it;
  if (relres) *relres = rel / scale;  // ||r0 - A d|| / ||b||
  return s;
}

}  // namespace gabp
