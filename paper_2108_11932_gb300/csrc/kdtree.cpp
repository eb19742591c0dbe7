// KD-tree ordering of the points into tiles (Section 6, clustering paragraph).
// A cluster of n > b points is sorted along the axis of largest bounding-box
// extent (ties: lowest axis), by (coordinate, original index), and split into a
// left cluster of b * 2^(ceil(log2(n/b)) - 1) points and a right cluster with
// the rest; a cluster of n <= b points is a leaf and keeps its order.  All
// leaves then hold b points except possibly the last one.
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace tlr {

static int64_t left_size(int64_t n, int b) {
  int64_t t = b;
  while (t < n) t <<= 1;  // smallest b * 2^p >= n
  return t >> 1;
}

static void rec(const double* x, int d, int b, int64_t* idx, int64_t n) {
  while (n > b) {
    double lo[3], hi[3];
    for (int q = 0; q < d; ++q) { lo[q] = x[idx[0] * d + q]; hi[q] = lo[q]; }
    for (int64_t p = 1; p < n; ++p)
      for (int q = 0; q < d; ++q) {
        const double v = x[idx[p] * d + q];
        lo[q] = std::min(lo[q], v);
        hi[q] = std::max(hi[q], v);
      }
    int ax = 0;
    double best = hi[0] - lo[0];
    for (int q = 1; q < d; ++q)
      if (hi[q] - lo[q] > best) { best = hi[q] - lo[q]; ax = q; }
    std::sort(idx, idx + n, [&](int64_t a, int64_t c) {
      const double va = x[a * d + ax], vc = x[c * d + ax];
      return va < vc || (va == vc && a < c);
    });
    const int64_t nl = left_size(n, b);
    rec(x, d, b, idx, nl);
    idx += nl;
    n -= nl;
  }
}

void kd_order(const double* pts, int64_t N, int d, int b, int64_t* perm) {
  for (int64_t p = 0; p < N; ++p) perm[p] = p;
  if (N > 0) rec(pts, d, b, perm, N);
}

}  // namespace tlr
