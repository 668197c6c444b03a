// Position of a frequency's representative in the half-grid list (host and device).
//
// The half grid keeps f = j m + l when f <= fc, fc = ((n - j) mod n) m + (m - l) mod m (the
// conjugate frequency of a real kernel's symbol), in increasing order. Row by row that is:
// row 0 and, for even n, row n/2 keep l = 0 .. floor(m/2) (there fc lies in the same row);
// rows 1 .. ceil(n/2) - 1 keep every l (fc lies in a later row); later rows keep none.
#pragma once

#include <cuda_runtime.h>

namespace lfa {

__host__ __device__ __forceinline__ int half_position(int n, int m, int f) {
  int j = f / m, l = f - j * m;
  const int jc = j == 0 ? 0 : n - j, lc = l == 0 ? 0 : m - l;
  if (jc * m + lc < f) { j = jc; l = lc; }      // the representative is the conjugate
  const int row0 = m / 2 + 1;                   // entries kept in row 0 (and in row n/2)
  if (j == 0) return l;
  return row0 + (j - 1) * m + l;                // rows 1 .. ceil(n/2)-1 full; row n/2 a prefix
}

}  // namespace lfa
