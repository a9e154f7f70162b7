// cluster.cuh -- the sums of a round run by one thread-block cluster, the same
// bits in every thread of the cluster, so every CTA takes the same decision after
// one cluster barrier.
#pragma once

#include <cooperative_groups.h>

#include "devutil.cuh"

namespace gabp {

struct __align__(16) ClusterPart {
  double rr;  // a warp's sum of its lanes' squared residuals
  int flags;  // the warp's flags, or-ed (their meaning is the kernel's)
  int pad;
};
struct ClusterSums {
  double rr;
  int flags;
};
// The sums of a cluster round, the same bits in every thread of the cluster: each warp adds its
// lanes' residual terms by an xor butterfly (at every step a lane and its partner add the same two
// values, so all lanes end equal) and lane 0 posts the sum in its CTA's shared memory; after the
// cluster barrier lane l of every warp adds the posts of warps l, l + 32, ... in that order (warp
// w of CTA r is warp NW r + w) and a second butterfly adds the lanes.  The flags are or-ed.
template <int NW>
__device__ __forceinline__ ClusterSums cluster_sums(cooperative_groups::cluster_group &cl, ClusterPart *part,
                                                    double rr, int flags, int lane, int wib, int nwarps) {
  const double w = warp_sum(rr);
  const int f = (int)__reduce_or_sync(0xffffffffu, (unsigned)flags);
  if (lane == 0) {
    part[wib].rr = w;
    part[wib].flags = f;
  }
  cl.sync();
  double x = 0.0;
  unsigned g = 0;
  for (int v = lane; v < nwarps; v += 32) {
    const ClusterPart *q = cl.map_shared_rank(part + v % NW, (unsigned)(v / NW));
    x += q->rr;
    g |= (unsigned)q->flags;
  }
  return ClusterSums{warp_sum(x), (int)__reduce_or_sync(0xffffffffu, g)};
}

// Two sums of a cluster round in the same way, the same bits in every thread (no flags).
struct __align__(16) ClusterPart2 {
  double a, b;
};
template <int NW>
__device__ __forceinline__ double2 cluster_sums2(cooperative_groups::cluster_group &cl, ClusterPart2 *part,
                                                 double a, double b, int lane, int wib, int nwarps) {
  const double wa = warp_sum(a), wb = warp_sum(b);
  if (lane == 0) {
    part[wib].a = wa;
    part[wib].b = wb;
  }
  cl.sync();
  double x = 0.0, y = 0.0;
  for (int v = lane; v < nwarps; v += 32) {
    const ClusterPart2 *q = cl.map_shared_rank(part + v % NW, (unsigned)(v / NW));
    x += q->a;
    y += q->b;
  }
  return make_double2(warp_sum(x), warp_sum(y));
}

}  // namespace gabp
