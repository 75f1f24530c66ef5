// Key-indexed start values: the first output of a SplitMix64 stream
// (Steele, Lea and Flood, OOPSLA 2014) whose state is seed ^ key, top 53
// bits mapped to a double in [-1, 1).
#pragma once

namespace edk {

__device__ __forceinline__ double splitmix_value(unsigned long long seed, unsigned long long key) {
  unsigned long long z = (seed ^ key) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

}  // namespace edk
