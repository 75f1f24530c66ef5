// Device helpers shared by the batched kernels.
#pragma once

namespace edk {

// index i with pref[i] <= v < pref[i + 1] (pref ascending, n entries used)
__device__ __forceinline__ int find_pref(const long long* pref, int n, long long v) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace edk
