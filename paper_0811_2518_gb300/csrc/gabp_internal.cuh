// gabp_internal.cuh -- device data layout and host-side handle of the GaBP solver.
//
// Layout in HBM (all arrays owned by the handle):
//   off-diagonal CSR in receiver layout: row i, slot e in [rp[i], rp[i+1]) with
//   k = ci[e] holds the message k -> i.  av[e] = A_ik, ad[i] = A_ii.
//   rev[e] is the slot of the reverse edge (row k, column i).
//   FP64 path: M64[2][E] double2 {P, h} (h = P * mu, the information form of the
//   mean message), N64[2][n] 32-byte node records {P~, h~, x, -}.
//   FP32 path: precision chains MP[2][E] float, coefficient pairs CF[E] float2,
//   mean chains H[2][E][R] float, node rings.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <cstdint>
#include <cstddef>
#include <functional>
#include <string>
#include <vector>
#include <algorithm>
#include <cmath>

#include "../../include/gabp.h"

namespace gabp {

constexpr int kBlock = 256;

struct __align__(32) NodeRec64 {
  double P;  // P~_i = A_ii + sum_k P_ki
  double h;  // h~_i = b_i + sum_k h_ki
  double x;  // x_i = h~_i / P~_i
  double pad;
};

// Device-side control block of one iterative run.  Written by the last block
// of each round kernel; every round kernel reads it first.
struct DevCtl {
  int round;         // last completed round t
  int done;          // 1 once a terminal decision was taken
  int status;        // gabp_status of the run
  int iters;         // rounds of the returned iterate (or at which breakdown happened)
  int result_round;  // round whose node records hold the answer
  int max_iter;
  int check_from;    // first round whose iterate may be accepted (1 for GaBP)
  int stable;        // consecutive rounds with a stationary precision set
  double bb;         // ||b||^2
  double tol2bb;     // tol^2 ||b||^2
  double rr;         // squared residual (or squared update) of the latest checked iterate
  double maxrel;     // FP32 precision rounds: messages that moved by more than 2^-s in the latest round
  double xx;         // squared norm of the latest iterate (FP32 inner solves)
  unsigned int arrive;
  int edge_bad;      // breakdown flag raised by an edge kernel, consumed by the round's last block
  const double *b;   // right-hand side of the current FP64 run (device); read by the round kernels
  int no_stop;       // autotuning runs: advance rounds but never take a terminal decision
  int hist_cap;      // FP64 rounds: entries of hist (0 = no history)
  double *hist;      // FP64 rounds: squared residual of iterate t at hist[t] (device, hist_cap entries)
  int hist_len;      // entries written
  int lam_round;     // Steffensen: the round whose extrapolation was applied last
  double lam;        // Steffensen: scalar step of the latest cycle (its second round's last block)
  int fstate;        // FP64 precision freeze: 0 screen, 1 verify and store the coefficients, 2 frozen
  int pstat;         // FP64 precision freeze: consecutive screened rounds with no aggregate moving
  int fround;        // FP64 precision freeze: the round that stored the coefficients (0: not yet)
  int pfail;         // FP64 precision freeze: failed verifications
  int fchecks;       // FP64 precision freeze: verification rounds run
  int fmove;         // FP64 precision freeze, serial schedule: raised by a sweep's kernels when a
                     // screened aggregate or a verified message moved; consumed by the decision
};

// Precision freeze (options.freeze_precisions).  The precision messages do not
// depend on b and converge on their own; once they have stopped moving (to
// rounding) the coefficients c = -A / P_k\i are constant and later rounds need
// only the mean messages.  States (fs, the state a round ran in):
//   0 screen: every node's P~_i is compared with its previous round's; after
//     2 << min(failed verifications, 5) consecutive rounds in which none moved,
//     the next round verifies;
//   1 verify: every precision message is compared with its own previous round's
//     while the round stores its coefficients and 1/P~; if none moved the
//     precisions are frozen from the next round on, else back to screening (a
//     message can still move while every aggregate it enters is stagnant, where
//     a cavity P~_k - P_ik cancels; the longer screens bound the verify rounds);
//   2 frozen: mean messages only, with the stored coefficients.
// "Moved": more than 16 units in the last place apart (bit patterns as integers;
// about 2^-48 relative).  Stagnant precision messages still jitter by a few units
// in the last place (rounding of the sums and differences they come from, larger
// where P~_k = A_kk + sum of negative messages cancels), so a tighter bar may never
// pass; the mean iteration with coefficients this close to their limits stays
// within rounding of the plain iterate.
__device__ __forceinline__ void freeze_step(DevCtl *ctl, int fs, int t, double moving) {
  if (fs == 0) {
    ctl->pstat = moving == 0.0 ? ctl->pstat + 1 : 0;
    if (ctl->pstat >= (2 << min(ctl->pfail, 5))) ctl->fstate = 1;
  } else if (fs == 1) {
    ctl->fchecks += 1;
    if (moving == 0.0) {
      ctl->fstate = 2;
      ctl->fround = t;
    } else {
      ctl->fstate = 0;
      ctl->pstat = 0;
      ctl->pfail += 1;
    }
  }
}

// More than 16 units in the last place apart (any NaN, a sign change or a zero
// against a non-zero counts as apart; two equal bit patterns do not).
__device__ __forceinline__ bool ulp_apart(double u, double v) {
  return (unsigned long long)(__double_as_longlong(u) - __double_as_longlong(v) + 16) > 32ull;
}

struct Graph {
  int n = 0;
  int64_t nnz = 0;  // full CSR (with diagonal)
  int E = 0;        // off-diagonal entries = directed edges
  int *rowptr = nullptr, *col = nullptr;  // full CSR copy (device)
  double *val = nullptr;
  int *rp = nullptr, *ci = nullptr, *rev = nullptr, *dpos = nullptr;
  double *av = nullptr, *ad = nullptr;
  float *av32 = nullptr, *ad32 = nullptr;
  double avg_deg = 0;
};

// Sliced layout of the FP64 parallel rounds (solve64.cu).  Rows are ordered by
// degree (descending) inside windows of kSellWindow rows and cut into slices of 32;
// slot j of the 32 rows of slice s sits at sp[s] + 32 j + lane, so a warp reads
// and writes whole contiguous lines and its lanes (one row each) do equal work.
// Positions past a row's degree hold sender -1 (padding).
struct Sell64 {
  bool ready = false;
  bool vals_ok = false;  // sav matches the graph's values (cleared by gabp_set_values)
  int ns = 0;            // slices
  int Es = 0;            // positions (slots + padding)
  int *srow = nullptr;   // [ns * 32] row of each slice lane, -1 past n
  int *sp = nullptr;     // [ns + 1] first position of each slice
  int *sci = nullptr;    // [Es] sender, -1 for padding
  int *srev = nullptr;   // [Es] position of the reverse edge
  double *sav = nullptr; // [Es] A value
  int *c2s = nullptr;    // [E] position of compact CSR slot e
};

struct Work64 {
  double2 *M[2] = {nullptr, nullptr};  // messages at the sliced positions
  NodeRec64 *N[2] = {nullptr, nullptr};
  bool valid = false;   // a solve has completed; messages/records are readable
  int result_round = 0;
  Sell64 sl;
  unsigned *bar = nullptr;  // grid barrier of the cooperative rounds: arrivals, generation, error flag
  double *C = nullptr;      // [Es] frozen coefficients c = -A / (P~ - P) (options.freeze_precisions)
};

struct Work32 {
  // precision phase (recompute form): chains + node ring of 3
  float *MP[2] = {nullptr, nullptr};
  float *NP[3] = {nullptr, nullptr, nullptr};
  float2 *CF = nullptr;   // {c_in, c_out} per slot
  float *invP = nullptr;  // 1 / P~_i (frozen)
  bool coef_ready = false;
  int prec_round = -1;    // round of the frozen precision state
  int R = 0;              // RHS capacity of the mean buffers
  float *H[2] = {nullptr, nullptr};               // [E][R]
  float *NH[3] = {nullptr, nullptr, nullptr};     // [n][R] h~ ring
  float *rhs32 = nullptr;                         // [n][R]
  double *X = nullptr, *Rs = nullptr;             // [n][R] FP64 iterate and residual
  double *Bt = nullptr;                           // [n][R] FP64 right-hand sides (interleaved)
  double *colnorm = nullptr;                      // per-RHS reductions [4][R]
  DevCtl *ctlR = nullptr;                         // per-RHS control (refinement)
  int *rhs_active = nullptr;
  float2 *NQ[3] = {nullptr, nullptr, nullptr};    // [n] {P~, h~} ring of the joint rounds
  struct RefineCtl *rc = nullptr;                 // device-resident refinement loop state
  struct RefineCtl *rc_host = nullptr;            // pinned copy read after a device-loop solve
  double *Bd = nullptr;                           // [n] right-hand side staged for the device loop
};

// Serial schedule (serial.cu): colouring, colour-grouped relabelling,
// colour-sorted slot layout, state.
struct WorkS {
  bool ready = false;
  int C = 0;                   // number of colours
  std::vector<int> cstart;     // [C+1] first new label of each colour class (host)
  int *colour = nullptr;       // [n] colour of each node (input labels)
  int *oid = nullptr;          // [n] new label -> input label
  int *nid = nullptr;          // [n] input label -> new label
  int *srp = nullptr;          // [n+1] row pointer of the new rows
  int *scol = nullptr;         // [n] colour of each new row
  int *co = nullptr;           // [(C+1) x n] segment bounds per colour
  int *sperm = nullptr;        // [E] serial slot -> input-layout slot
  int *sci = nullptr;          // [E] sender (new label) of a serial slot
  int *srev = nullptr;         // [E] serial slot of the reverse edge
  double *sav = nullptr;       // [E] A values in serial order
  double *sad = nullptr;       // [n] A_jj in the new order
  double *sb = nullptr;        // [n] b in the new order (FP64 sweeps)
  double *bin = nullptr, *xin = nullptr;  // [n] staged b and iterate (input order) of the FP64 sweeps
  double2 *SM = nullptr;       // [E] FP64 messages {P, h}
  double2 *fire = nullptr;     // [n] FP64 firing aggregates
  double *sPm = nullptr;       // [n] marginal precisions of the last FP64 sweep (new order)
  double *sh1 = nullptr;       // [E] Steffensen: mean messages after a cycle's first sweep
  double *sx0 = nullptr, *sx1 = nullptr;  // [n] Steffensen: iterates x_n, x_{n+1} (input order)
  double *coef = nullptr;      // [E] precision freeze: coefficients -A_kj / P_k\j in the serial order
  int *dcstart = nullptr;      // [C+1] cstart on the device (the one-cluster sweeps)
  std::vector<int> srp_h;      // [n+1] srp on the host (sizes of the on-chip sweeps)
  int clu = -1;                // CTAs of the one-cluster FP64 sweeps (0: none; -1: not yet sized)
  int clu_nw = 0;              // warps per CTA there
  int chip_bytes = 0;          // shared memory a CTA of those sweeps with the state on chip (0: no fit)
  int chip_bytes_stf = 0;      // the same with Steffensen's step
  int chip_S = 0;              // slots of the largest CTA there
  bool valid = false;
  int result_round = 0;
  float2 *sCF = nullptr;       // [E] frozen coefficients in serial order
  float *sH = nullptr;         // [E] FP32 mean messages
  float *hfire = nullptr;      // [n] FP32 firing aggregates h~
  float *srhs = nullptr;       // [n] inner right-hand side (new order)
  float *sinvP = nullptr;      // [n] 1 / P~ (new order)
};

// Sliced layout of the independent-systems grid kernel: every system's rows sorted by
// degree (descending, stable) in windows of 4096 and cut into 32-row slices, the last
// slice of a system padded with rows -1, so that a slice belongs to one system; slot j
// of the slice's rows is the contiguous line sp[s] + 32 j + lane (sender -1 past a
// row's degree).  Built for one offsets array; the values are refreshed after
// gabp_set_values.
struct GSell {
  std::vector<int> off;        // the offsets the layout was built for
  int ns = 0;                  // slices
  int Es = 0;                  // slots, padding included
  bool vals_ok = false;
  int *srow = nullptr;         // [32 ns] row of each slice lane, -1 for padding
  int *sp = nullptr;           // [ns + 1] first slot of each slice (multiples of 32)
  int *ssys = nullptr;         // [ns] system of each slice
  int *sci = nullptr;          // [Es] sender, -1 for padding
  float *sav = nullptr;        // [Es] A_ij (FP32), 0 for padding
  float *MP[2] = {nullptr, nullptr}, *H[2] = {nullptr, nullptr};  // [Es] precision / mean chains
  float2 *CF = nullptr;        // [Es] frozen coefficients
};

// Single-loop convergence fix (fixloop.cu)
struct WorkF {
  double2 *M[2] = {nullptr, nullptr};
  double2 *N[2] = {nullptr, nullptr};
  double *hpot = nullptr, *bin = nullptr, *xin = nullptr;
  double step = 0.0;  // damping step the cached round graph was captured with
};

struct WorkB;  // batched multi-RHS work arrays (batched.cu)

struct Stats {
  int64_t rounds = 0;
  int64_t edge_updates = -1;  // set by paths whose systems differ in size (else rounds x E x nrhs)
  int refine_steps = 0;
  int nrhs = 1;
  int freeze_round = 0;   // FP64 precision freeze: the round whose coefficients were stored (0: none)
  int freeze_checks = 0;  // FP64 precision freeze: verification rounds run
};

// Phase timing (options.profile): CUDA events around each phase's launches.
enum { PH_FP64 = 0, PH_PREC32 = 1, PH_MEAN32 = 2, PH_REFINE64 = 3, PH_MULTI = 4, PH_FREEZE32 = 5, PH_COUNT = 6 };
struct Prof {
  double ms[PH_COUNT] = {0, 0, 0, 0, 0, 0};
  int64_t rounds[PH_COUNT] = {0, 0, 0, 0, 0, 0};
  int64_t launches = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

}  // namespace gabp

struct gabp_handle_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  // When the caller gives no stream (the legacy default stream), the handle runs on a stream of
  // its own -- round graphs cannot be captured on the legacy stream -- ordered after the caller's
  // default-stream work at every entry point (order_after_caller).
  cudaStream_t own_stream = nullptr;
  cudaEvent_t caller_ev = nullptr;
  bool order_legacy = false;
  gabp_options opt{};
  gabp::Graph g;
  gabp::Work64 w64;
  gabp::Work32 w32;
  gabp::Stats stats;
  gabp::DevCtl *ctl = nullptr;      // device control block
  gabp::DevCtl *ctl_host = nullptr; // pinned mirror
  double *partials = nullptr;       // per-block partial sums [4 * max_blocks]
  int max_blocks = 0;
  int num_sms = 0;
  double *hb = nullptr, *hx = nullptr;  // device staging for gabp_solve_host
  // captured round graphs (keyed by kind), rebuilt when options change
  cudaGraphExec_t g64 = nullptr;
  int g64_key = -1;
  cudaGraphExec_t gP32 = nullptr;
  cudaGraphExec_t gH32 = nullptr;
  cudaGraphExec_t gJ32 = nullptr;   // joint precision + mean rounds
  gabp::WorkS ws;                   // serial schedule
  gabp::WorkF wf;                   // single-loop convergence fix
  cudaGraphExec_t gSL = nullptr;
  long long gSL_key = -1;
  cudaGraphExec_t gS64 = nullptr, gS32 = nullptr;  // serial sweeps (FP64, FP32 mean)
  long long gS64_key = -1, gS32_key = -1;
  cudaGraph_t gRefG = nullptr;      // whole FP32 refinement loop (conditional nodes) and its instance
  cudaGraphExec_t gRef = nullptr;
  long long gRef_key = -1;
  long long gJ32_L = -1;
  int tuned_Lj32 = 0;               // autotuned shape of the joint round
  int gH32_R = -1;
  int last_path = -1;               // 0 FP64, 1 FP32 refinement (for gabp_marginal_precisions)
  // autotuned sub-warp widths (0 = not tuned yet) and the scratch control block the tuner uses
  int tuned_L64 = 0, tuned_Lp32 = 0, tuned_Lm32 = 0;
  gabp::DevCtl *ctl_tune = nullptr;
  long long gP32_L = -1, gH32_L = -1;
  double *gamma = nullptr;          // diagonal loading of the convergence fix (device, n)
  double *hist = nullptr;           // residual history of the last FP64 run (device, opt.history entries)
  int hist_alloc = 0;
  int hist_len = 0;                 // entries recorded by the last solve (0 when it kept none)
  double hist_bb = 0.0;             // ||b||^2 of that solve
  double *ig_buf = nullptr;         // initial-guess solves: r0 = b - A x0, the correction d, sums
  gabp::Prof prof;
  gabp::WorkB *wb = nullptr;
  long long multi_big = 0;          // autotuned cluster / single-CTA size split of the multi-system kernel
  int multi_nt = 0;                 // autotuned block size of the multi-system kernel
  bool values_ok = true;            // false after a rejected gabp_set_values
  int multi_mode = 0;               // 0 untuned, 1 grid-persistent kernel, 2 cluster / single-block teams
  int multi_grid_shape = 0;         // autotuned shape of the grid-persistent kernel (0 untuned)
  gabp::GSell *gsl = nullptr;       // sliced layout of the grid-persistent kernel (built on first use)
  // least squares (gabp_create_lsq): the handle's matrix is [[I_k, J^T], [J, -gamma I_m]]
  int clu64 = 0;                    // CTAs of the FP64 cluster rounds (0: graph too large or no support)
  int clu64_nw = 0;                 // warps per CTA there (2 or 4)
  int chip64_bytes = 0;             // shared memory per CTA of those rounds with all state on chip (0: no fit)
  int chip64_smax = 0, chip64_rmax = 0;  // own slots and own rows of the largest CTA there
  int coop64 = 0;                   // blocks of the FP64 cooperative rounds (0: graph too large or no support)
  int coop64f = 0;                  // the same for the cooperative rounds with the precision freeze
  int lsq_m = 0, lsq_k = 0;         // 0: not a least-squares handle
  double *lsq_b = nullptr, *lsq_x = nullptr;  // [k + m] augmented right-hand side and solution
};
namespace gabp {
// Orders the handle's own stream after the work the caller queued on the legacy
// default stream (its inputs, or earlier use of its output buffers); a no-op when
// the caller supplied a stream.
inline void order_after_caller(gabp_handle_s *h) {
  if (!h->order_legacy) return;
  cudaEventRecord(h->caller_ev, cudaStreamLegacy);
  cudaStreamWaitEvent(h->stream, h->caller_ev, 0);
}
}  // namespace gabp


namespace gabp {

// error plumbing ---------------------------------------------------------------
void set_last_error(const std::string &s);
// api.cu: pointer kind test (allocates nothing) and the single-RHS dispatcher of gabp_solve
bool is_device_ptr(const void *p);
bool values_usable(gabp_handle_s *h);
gabp_status solve_dispatch(gabp_handle_s *h, const double *b, double *x, double tol, int32_t max_iter,
                           int32_t *iters_out, double *relres_out);
gabp_status cuda_fail(cudaError_t e, const char *what);

#define GABP_CUDA(call)                                     \
  do {                                                      \
    cudaError_t e__ = (call);                               \
    if (e__ != cudaSuccess) return ::gabp::cuda_fail(e__, #call); \
  } while (0)

// Grid of one full wave: SMs x CTAs of this kernel resident per SM (grid-stride
// kernels then give every CTA the same share with no partial second wave).
template <typename K>
inline int resident_grid(int num_sms, K kernel) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kBlock, 0) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  return nb * num_sms;
}

inline int blocks_for(int64_t work, int per_block, int max_blocks) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

// Profiling brackets: prof_begin records e0 before a phase's launches,
// prof_end records e1 after them; prof_collect (after a synchronisation) adds
// the elapsed time to the phase.
inline void prof_begin(gabp_handle h) {
  if (h->opt.profile) cudaEventRecord(h->prof.e0, h->stream);
}
inline void prof_end(gabp_handle h) {
  if (h->opt.profile) cudaEventRecord(h->prof.e1, h->stream);
}
inline void prof_collect(gabp_handle h, int phase, int64_t rounds) {
  h->prof.rounds[phase] += rounds;
  if (!h->opt.profile) return;
  cudaEventSynchronize(h->prof.e1);  // profiling mode only: wait for the phase's end
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, h->prof.e0, h->prof.e1) == cudaSuccess) h->prof.ms[phase] += ms;
  else cudaGetLastError();
}

// Autotuner: times `rounds` launches of `launch` (after one warm-up launch) on
// the handle's stream; the caller points the kernels at a scratch control block
// with no_stop set, so the launches do real work whatever the buffers hold.
template <typename F>
inline float time_launches(gabp_handle h, F launch, int rounds) {
  // the fastest single launch (x rounds): robust to a neighbour's interference
  launch();
  constexpr int kMaxEv = 16;
  rounds = rounds < 1 ? 1 : (rounds > kMaxEv - 1 ? kMaxEv - 1 : rounds);
  cudaEvent_t ev[kMaxEv];
  int made = 0;
  for (; made <= rounds; ++made)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
  float best = 1e30f;
  if (made == rounds + 1) {
    cudaEventRecord(ev[0], h->stream);
    for (int r = 0; r < rounds; ++r) {
      launch();
      cudaEventRecord(ev[r + 1], h->stream);
    }
    if (cudaEventSynchronize(ev[rounds]) == cudaSuccess) {
      for (int r = 0; r < rounds; ++r) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[r], ev[r + 1]) == cudaSuccess && ms < best) best = ms;
      }
    }
  }
  cudaGetLastError();
  for (int j = 0; j < made; ++j) cudaEventDestroy(ev[j]);
  return best < 1e30f ? best * rounds : 1e30f;
}
gabp_status tune_ctl(gabp_handle h, const double *b);  // (re)arms ctl_tune for a tuning run (b: any n-vector)

gabp_status read_ctl(gabp_handle h);  // copies ctl -> ctl_host and synchronises

// Tolerance of one FP32 inner solve: only the reduction still needed to reach
// tol (with a factor 10 of margin), never looser than the option's inner_tol,
// never tighter than FP32 can deliver (1e-6) unless inner_tol itself asks for it.
__host__ __device__ inline double inner_target(double inner_tol, double tol, double bb, double rr) {
  const double need = rr > 0.0 ? 0.1 * tol * sqrt(bb / rr) : inner_tol;
  return fmin(inner_tol, fmax(1e-6, need));
}

// Run K-round graphs of one round kernel (CUDA graph of K launches when the
// stream can be captured) until the control block says done.
#define GABP_DISPATCH_L(L, CALL) \
  switch (L) {                   \
    case 1: { constexpr int LL = 1; CALL; } break;  \
    case 2: { constexpr int LL = 2; CALL; } break;  \
    case 4: { constexpr int LL = 4; CALL; } break;  \
    case 8: { constexpr int LL = 8; CALL; } break;  \
    case 16: { constexpr int LL = 16; CALL; } break; \
    default: { constexpr int LL = 32; CALL; } break; \
  }

template <typename LaunchFn>
inline gabp_status run_rounds(gabp_handle h, cudaGraphExec_t *cache, long long *cache_key, int key, LaunchFn launch,
                              int max_rounds, int phase, int round0 = 0) {
  const int K = h->opt.check_every;
  const bool use_graph = h->stream != nullptr && h->opt.graphs;
  // a cached graph holds K rounds of one launch shape: both are part of its key
  const long long full_key = ((long long)K << 32) | (unsigned)key;
  if (use_graph && *cache && *cache_key != full_key) {
    cudaGraphExecDestroy(*cache);
    *cache = nullptr;
  }
  if (use_graph && !*cache) {
    *cache_key = full_key;
    cudaGraph_t graph;
    GABP_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < K; ++k) launch();
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (e != cudaSuccess) return cuda_fail(e, "capture FP32 rounds");
    e = cudaGraphInstantiate(cache, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate FP32 rounds");
  }
  const int64_t max_batches = (int64_t)max_rounds / K + 3;
  int prev_round = round0;
  for (int64_t bI = 0; bI < max_batches; ++bI) {
    prof_begin(h);
    if (use_graph) {
      GABP_CUDA(cudaGraphLaunch(*cache, h->stream));
    } else {
      for (int k = 0; k < K; ++k) launch();
      GABP_CUDA(cudaGetLastError());
    }
    prof_end(h);
    h->prof.launches += K;
    gabp_status s = read_ctl(h);
    if (s != GABP_OK) return s;
    prof_collect(h, phase, h->ctl_host->round - prev_round);
    prev_round = h->ctl_host->round;
    if (h->ctl_host->done) return GABP_OK;
  }
  set_last_error("FP32 rounds ended without a decision");
  return GABP_ERR_CUDA;
}


// shared host helpers (defined in setup.cu / solve64.cu / solve32.cu)
// Process-wide memory of the autotuner's kernel shapes, keyed by (device, n,
// directed edges): a handle created for a matrix of the same size (typically the
// same pattern with new values, e.g. one handle per training step) starts tuned.
// An NVTX range over a solver phase (visible to ncu's --nvtx filters and timeline
// tools; a no-op unless a tool attaches).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Makes a device current for the scope of an entry point and restores the
// caller's device on exit (the handle's stream and memory live on its device).
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess) prev = cur;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard &) = delete;
  DeviceGuard &operator=(const DeviceGuard &) = delete;
};

void tune_cache_load(gabp_handle h);
int pinned_shape32(int lanes, int unroll);  // solve32.cu: shape code of a pinned (lanes, unroll), 0 if none
void tune_cache_store(gabp_handle h);
gabp_status ensure_w64(gabp_handle h);
void free_w64(gabp_handle h);
gabp_status ensure_w32(gabp_handle h, int R);
void free_w32(gabp_handle h);
gabp_status solve64(gabp_handle h, const double *b, double *x, double tol, int max_iter, int *iters,
                    double *relres);
gabp_status solve32_refine(gabp_handle h, int R, const double *B, double *X, int64_t ld, double tol,
                           int max_iter, const double *gamma_diag, int *iters, double *relres);
gabp_status messages64(gabp_handle h, double *P, double *hm);
gabp_status marginals(gabp_handle h, double *Pi);
gabp_status grad_values(gabp_handle h, const double *lam, const double *x, double *g);
gabp_status make_gamma(gabp_handle h, double *out);
gabp_status marginals32(gabp_handle h, double *Pi);
gabp_status precision_phase32(gabp_handle h, const double *gamma_diag);
void free_wb(gabp_handle h);
gabp_status solve_systems(gabp_handle h, int nsys, const int *offsets_host, const double *b, double *x, double tol,
                          int max_iter, int *status_host, int *iters_host, double *relres_host);
// single-loop convergence fix (fixloop.cu)
void free_wf(gabp_handle h);
gabp_status solve_fix_single(gabp_handle h, const double *b, double *x, double tol, int max_iter,
                             const double *gamma_diag, int *iters, double *relres);
// serial schedule (serial.cu)
void free_ws(gabp_handle h);
gabp_status serial_prepare(gabp_handle h);
gabp_status serial_colours(gabp_handle h, int *colour_dev, int *ncolours);
gabp_status serial_refresh_values(gabp_handle h);
gabp_status solve64_serial(gabp_handle h, const double *b, double *x, double tol, int max_iter, int *iters,
                           double *relres);
gabp_status serial_messages64(gabp_handle h, double2 *M_input_layout);
gabp_status serial_marginals64(gabp_handle h, double *Pi);
gabp_status serial_freeze32(gabp_handle h, const float2 *CF, const float *invP);
gabp_status serial_inner32(gabp_handle h, const float *rhs, int cap, double itol, int *sweeps, int *status);
gabp_status serial_update32(gabp_handle h, double *X);
gabp_status load_messages64(gabp_handle h, const double *P, const double *hm);
// initial.cu: x holds x0 on entry; solve(r0, d, tol', iters, relres) runs a path on A d = b - A x0
gabp_status solve_from_initial(gabp_handle h, const double *b, double *x, double tol, int *iters, double *relres,
                               const std::function<gabp_status(const double *, double *, double, int *, double *)>
                                   &solve);
gabp_status messages64_from(gabp_handle h, const double2 *M, double *P, double *hm);
// Shapes (lanes per row L | slots per lane U << 8) of the grid-persistent
// multi-system kernel the autotuner chooses from.
// kSliced marks the kernel on the sliced layout (GSell: one lane per row, U slots of a
// row issued together; L is 1).
constexpr int kSliced = 1 << 16;
constexpr int kGridShapes[12] = {1 | (4 << 8), 2 | (4 << 8), 4 | (2 << 8), 4 | (4 << 8), 8 | (2 << 8),
                                  1 | (2 << 8), 2 | (2 << 8), 1 | (1 << 8), 2 | (1 << 8),
                                  kSliced | 1 | (1 << 8), kSliced | 1 | (2 << 8), kSliced | 1 | (4 << 8)};
gabp_status solve_systems_grid(gabp_handle h, int nsys, const int *d_off, const int *off_host, const double *b,
                               double *x, double tol, int max_iter, int *d_status, int *d_iters, int *d_refine,
                               double *d_relres, int shape, float *ms_out);
void free_gsell(gabp_handle h);
gabp_status solve_batched32(gabp_handle h, int nrhs, const double *B, double *X, int64_t ld, double tol,
                            int max_iter, int *iters, double *relres_host);

}  // namespace gabp
