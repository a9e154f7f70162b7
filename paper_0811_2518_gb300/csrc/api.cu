// api.cu -- the C ABI entry points that run solves (gabp_create / gabp_destroy /
// options / status strings live in setup.cu).
#include "gabp_internal.cuh"

#include <algorithm>
#include <cmath>

using namespace gabp;

namespace gabp {

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// a handle whose last gabp_set_values was rejected holds no valid matrix
bool values_usable(gabp_handle h) {
  if (h->values_ok) return true;
  set_last_error("the handle's values were rejected by gabp_set_values; set valid values first");
  return false;
}

gabp_status solve_dispatch(gabp_handle h, const double *b, double *x, double tol, int32_t max_iter,
                           int32_t *iters_out, double *relres_out) {
  if (!h || !b || !x || !(tol >= 0.0) || max_iter < 0 || !values_usable(h)) return GABP_ERR_INVALID;
  DeviceGuard dg(h->device);
  order_after_caller(h);
  h->hist_len = 0;  // only the FP64 parallel rounds record a history
  h->stats.freeze_round = h->stats.freeze_checks = 0;  // and only they freeze on the device
  // one solve of A x = b on the path the options select (x = 0 at the start)
  auto run = [&](const double *rb, double *rx, double rtol, int *it, double *rel) -> gabp_status {
    gabp_status s;
    if (h->opt.gamma_mode != 0) {
      // convergence fix: FP32 GaBP inner solves on A + Gamma inside the FP64 outer loop
      if (!h->gamma) {
        cudaError_t e = cudaMalloc(&h->gamma, sizeof(double) * h->g.n);
        if (e != cudaSuccess) return cuda_fail(e, "gamma");
      }
      s = make_gamma(h, h->gamma);
      if (h->opt.fix_single_loop) {
        if (s == GABP_OK) s = solve_fix_single(h, rb, rx, rtol, max_iter, h->gamma, it, rel);
        h->last_path = -1;  // the messages are those of A + Gamma: no marginals of A to report
      } else {
        if (s == GABP_OK) s = solve32_refine(h, 1, rb, rx, h->g.n, rtol, max_iter, h->gamma, it, rel);
        h->last_path = 1;
      }
    } else if (h->opt.precision == GABP_PREC_FP32_REFINE) {
      s = solve32_refine(h, 1, rb, rx, h->g.n, rtol, max_iter, nullptr, it, rel);
      h->last_path = 1;
    } else if (h->opt.schedule == 1) {
      s = solve64_serial(h, rb, rx, rtol, max_iter, it, rel);
      h->last_path = 2;
    } else {
      s = solve64(h, rb, rx, rtol, max_iter, it, rel);
      h->last_path = 0;
    }
    return s;
  };
  int it = 0;
  double rel = 0.0;
  gabp_status s;
  if (h->opt.initial_guess) {
    s = solve_from_initial(h, b, x, tol, &it, &rel, run);
  } else {
    s = run(b, x, tol, &it, &rel);
  }
  if (s >= 0) {
    if (iters_out) *iters_out = it;
    if (relres_out) *relres_out = rel;
  }
  return s;
}

}  // namespace gabp

extern "C" gabp_status gabp_solve(gabp_handle h, const double *b, double *x, double tol, int32_t max_iter,
                                  int32_t *iters_out, double *relres_out) {
  if (!h || !b || !x) return GABP_ERR_INVALID;
  if (!is_device_ptr(b) || !is_device_ptr(x)) {
    set_last_error("gabp_solve: b and x must be device arrays (use gabp_solve_host for host arrays)");
    return GABP_ERR_INVALID;
  }
  return solve_dispatch(h, b, x, tol, max_iter, iters_out, relres_out);
}

extern "C" gabp_status gabp_solve_host(gabp_handle h, const double *b, double *x, double tol, int32_t max_iter,
                                       int32_t *iters_out, double *relres_out) {
  if (!h || !b || !x) return GABP_ERR_INVALID;
  DeviceGuard dg(h->device);
  order_after_caller(h);
  const size_t bytes = sizeof(double) * h->g.n;
  if (!h->hb) {
    cudaError_t e = cudaMalloc(&h->hb, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "gabp_solve_host staging");
  }
  if (!h->hx) {
    cudaError_t e = cudaMalloc(&h->hx, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "gabp_solve_host staging");
  }
  GABP_CUDA(cudaMemcpyAsync(h->hb, b, bytes, cudaMemcpyHostToDevice, h->stream));
  if (h->opt.initial_guess)  // x holds the initial iterate
    GABP_CUDA(cudaMemcpyAsync(h->hx, x, bytes, cudaMemcpyHostToDevice, h->stream));
  gabp_status s = solve_dispatch(h, h->hb, h->hx, tol, max_iter, iters_out, relres_out);
  if (s < 0) return s;
  GABP_CUDA(cudaMemcpyAsync(x, h->hx, bytes, cudaMemcpyDeviceToHost, h->stream));
  GABP_CUDA(cudaStreamSynchronize(h->stream));
  return s;
}

extern "C" gabp_status gabp_solve_batched(gabp_handle h, int32_t nrhs, const double *B, double *X, int64_t ld,
                                          double tol, int32_t max_iter, int32_t *iters_out, double *relres_out) {
  if (!h || !B || !X || nrhs < 1 || ld < h->g.n || !(tol >= 0.0) || max_iter < 0 || !values_usable(h))
    return GABP_ERR_INVALID;
  if (!is_device_ptr(B) || !is_device_ptr(X)) {
    set_last_error("gabp_solve_batched: B and X must be device arrays");
    return GABP_ERR_INVALID;
  }
  DeviceGuard dg(h->device);
  order_after_caller(h);
  h->stats.freeze_round = h->stats.freeze_checks = 0;
  int it = 0;
  gabp_status s = solve_batched32(h, nrhs, B, X, ld, tol, max_iter, &it, relres_out);
  if (s >= 0 && iters_out) *iters_out = it;
  return s;
}

extern "C" gabp_status gabp_marginal_precisions(gabp_handle h, double *Pi) {
  if (!h || !Pi) return GABP_ERR_INVALID;
  DeviceGuard dg(h->device);
  order_after_caller(h);
  if (h->last_path == 0) return marginals(h, Pi);
  if (h->last_path == 1) return marginals32(h, Pi);
  if (h->last_path == 2) return serial_marginals64(h, Pi);
  return GABP_ERR_INVALID;
}

extern "C" gabp_status gabp_get_messages(gabp_handle h, double *P, double *hm) {
  if (!h || !P || !hm) return GABP_ERR_INVALID;
  DeviceGuard dg(h->device);
  order_after_caller(h);
  if (h->last_path == 0) return messages64(h, P, hm);
  if (h->last_path != 2) return GABP_ERR_INVALID;
  double2 *M = nullptr;  // serial messages back in the input layout
  GABP_CUDA(cudaMalloc(&M, sizeof(double2) * (size_t)(h->g.E > 0 ? h->g.E : 1)));
  gabp_status s = serial_messages64(h, M);
  if (s == GABP_OK) s = messages64_from(h, M, P, hm);
  cudaFree(M);
  return s;
}

extern "C" gabp_status gabp_set_messages(gabp_handle h, const double *P, const double *hm) {
  if (!h || !P || !hm || !values_usable(h)) return GABP_ERR_INVALID;
  if (!is_device_ptr(P) || !is_device_ptr(hm)) {
    set_last_error("gabp_set_messages: P and hm must be device arrays");
    return GABP_ERR_INVALID;
  }
  DeviceGuard dg(h->device);
  order_after_caller(h);
  gabp_status s = load_messages64(h, P, hm);
  h->last_path = -1;  // marginals and messages are reported again after the next solve
  return s;
}

extern "C" gabp_status gabp_serial_colours(gabp_handle h, int32_t *colour, int32_t *ncolours) {
  if (!h || !values_usable(h)) return GABP_ERR_INVALID;
  if (colour && !is_device_ptr(colour)) {
    set_last_error("gabp_serial_colours: colour must be a device array");
    return GABP_ERR_INVALID;
  }
  DeviceGuard dg(h->device);
  order_after_caller(h);
  return serial_colours(h, colour, ncolours);
}

extern "C" gabp_status gabp_grad_values(gabp_handle h, const double *lambda, const double *x, double *grad_val) {
  if (!h || !lambda || !x || !grad_val || !values_usable(h)) return GABP_ERR_INVALID;
  DeviceGuard dg(h->device);
  order_after_caller(h);
  return grad_values(h, lambda, x, grad_val);
}

extern "C" gabp_status gabp_last_stats(gabp_handle h, int64_t *rounds, int64_t *num_edges, int64_t *edge_updates,
                                       int32_t *refine_steps) {
  if (!h) return GABP_ERR_INVALID;
  if (rounds) *rounds = h->stats.rounds;
  if (num_edges) *num_edges = h->g.E;
  if (edge_updates)
    *edge_updates = h->stats.edge_updates >= 0 ? h->stats.edge_updates : h->stats.rounds * (int64_t)h->g.E;
  if (refine_steps) *refine_steps = h->stats.refine_steps;
  return GABP_OK;
}

extern "C" gabp_status gabp_last_freeze(gabp_handle h, int32_t *round, int32_t *checks) {
  if (!h) return GABP_ERR_INVALID;
  if (round) *round = h->stats.freeze_round;
  if (checks) *checks = h->stats.freeze_checks;
  return GABP_OK;
}

extern "C" gabp_status gabp_solve_systems(gabp_handle h, int32_t nsys, const int32_t *offsets, const double *b,
                                          double *x, double tol, int32_t max_iter, int32_t *status_out,
                                          int32_t *iters_out, double *relres_out) {
  if (!h || !offsets || !b || !x || nsys < 1 || !(tol >= 0.0) || max_iter < 0 || !values_usable(h))
    return GABP_ERR_INVALID;
  if (!is_device_ptr(b) || !is_device_ptr(x)) {
    set_last_error("gabp_solve_systems: b and x must be device arrays");
    return GABP_ERR_INVALID;
  }
  DeviceGuard dg(h->device);
  order_after_caller(h);
  h->stats.freeze_round = h->stats.freeze_checks = 0;
  return solve_systems(h, nsys, offsets, b, x, tol, max_iter, status_out, iters_out, relres_out);
}

extern "C" gabp_status gabp_profile_read(gabp_handle h, gabp_profile *out, int reset) {
  if (!h) return GABP_ERR_INVALID;
  if (out) {
    for (int j = 0; j < PH_COUNT; ++j) {
      out->ms[j] = h->prof.ms[j];
      out->rounds[j] = h->prof.rounds[j];
    }
    out->launches = h->prof.launches;
  }
  if (reset) {
    for (int j = 0; j < PH_COUNT; ++j) {
      h->prof.ms[j] = 0.0;
      h->prof.rounds[j] = 0;
    }
    h->prof.launches = 0;
  }
  return GABP_OK;
}

extern "C" gabp_status gabp_residual_history(gabp_handle h, double *relres, int32_t cap, int32_t *count) {
  if (!h || cap < 0 || (cap > 0 && !relres)) return GABP_ERR_INVALID;
  DeviceGuard dg(h->device);
  order_after_caller(h);
  const int m = std::min(cap, h->hist_len);
  if (m > 0) {
    GABP_CUDA(cudaMemcpyAsync(relres, h->hist, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, h->stream));
    GABP_CUDA(cudaStreamSynchronize(h->stream));
    for (int j = 0; j < m; ++j) relres[j] = h->hist_bb > 0.0 ? std::sqrt(relres[j] / h->hist_bb) : 0.0;
  }
  if (count) *count = h->hist_len;
  return GABP_OK;
}

extern "C" gabp_status gabp_tuned_shapes(gabp_handle h, int32_t *fp64_lanes, int32_t *prec32_shape,
                                         int32_t *mean32_shape, int64_t *multi_split, int32_t *multi_mode) {
  if (!h) return GABP_ERR_INVALID;
  if (fp64_lanes) *fp64_lanes = h->tuned_L64;
  if (prec32_shape) *prec32_shape = h->opt.overlap_precision ? h->tuned_Lj32 : h->tuned_Lp32;
  if (mean32_shape) *mean32_shape = h->tuned_Lm32;
  if (multi_split) *multi_split = h->multi_big;
  if (multi_mode) *multi_mode = h->multi_mode | (h->multi_grid_shape << 8);
  return GABP_OK;
}
