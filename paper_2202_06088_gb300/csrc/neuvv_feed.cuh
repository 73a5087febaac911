// Per-lane ray feed for the persistent kernels.
//
// A warp takes chunks of consecutive ray indices from a global counter (one
// atomic per chunk); a lane whose ray has finished takes the next index of the
// warp's chunk, so lanes do not idle while the longest ray of a packet
// finishes, and rays that miss the tree cost only their setup.
#pragma once

#include <cuda_runtime.h>

namespace neuvv {

struct WarpFeed {
  long long next, end;  // warp-uniform: unread part of the current chunk
  bool exhausted;       // warp-uniform: the counter has passed n
};

// One round of refilling: `need` is the ballot of lanes without a ray.  Takes
// a new chunk from the counter when the warp's chunk is used up and returns
// the ray index for the calling lane if it is needy and the chunk has one,
// else -1.  Sets f.exhausted when the counter has passed n.  All 32 lanes of
// the warp must call this together.
__device__ __forceinline__ long long feed_take(WarpFeed &f, unsigned long long *work, long long n, int chunk,
                                               unsigned need) {
  const int lane = threadIdx.x & 31;
  if (f.next >= f.end) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(work, (unsigned long long)chunk);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    f.next = (long long)base;
    f.end = f.next + chunk < n ? f.next + chunk : n;
    if (f.next >= n) {
      f.exhausted = true;
      return -1;
    }
  }
  const int rank = __popc(need & ((1u << lane) - 1u));
  const long long mine = f.next + rank;
  const long long taken = f.next + __popc(need);
  const long long end = f.end;
  f.next = taken < end ? taken : end;
  return ((need >> lane) & 1u) && mine < end ? mine : -1;
}

}  // namespace neuvv
