// Insertion orders (Sec. 5): the birth order a cloud is built in decides its
// successor lists, so it changes build time and query work but never the
// answers. Three orders, all deterministic for a given seed:
//   random        a seeded uniform permutation;
//   brio_hilbert  biased randomized insertion: a seeded permutation cut into
//                 rounds of doubling size (the last round half the points),
//                 each round sorted along a 3D Hilbert curve over the bounding
//                 box (the kind of spatial sort the paper's builder applies);
//   fpo           farthest-point order: each next point is the one whose
//                 distance to the points already taken is largest (ties to the
//                 lower input index), starting from input index 0.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <queue>
#include <string>
#include <vector>

#include "../../include/mknn.h"
#include "cloud.h"

namespace mknn {

namespace {

mknn_status ofail(mknn_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Seeded permutation: argsort of counter-based random keys.
std::vector<int64_t> random_permutation(int64_t n, uint64_t seed) {
  std::vector<std::pair<uint64_t, int64_t>> key((size_t)n);
  const uint64_t base = mix64(seed * 0x9E3779B97F4A7C15ULL + 0x5EEDULL);
  for (int64_t i = 0; i < n; ++i)
    key[i] = {mix64(base + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL), i};
  std::sort(key.begin(), key.end());
  std::vector<int64_t> out((size_t)n);
  for (int64_t i = 0; i < n; ++i) out[i] = key[i].second;
  return out;
}

}  // namespace

// Hilbert index of a cell of the 2^bits-per-axis grid: the axes are turned
// into the curve's transposed form by Skilling's method (Programming the
// Hilbert curve, AIP Conf. Proc. 707, 2004), then the transposed bits are
// interleaved, most significant first.
uint64_t hilbert_index3(uint32_t x, uint32_t y, uint32_t z, int bits) {
  uint32_t X[3] = {x, y, z};
  const uint32_t top = 1u << (bits - 1);
  for (uint32_t q = top; q > 1; q >>= 1) {
    const uint32_t low = q - 1;
    for (int i = 0; i < 3; ++i) {
      if (X[i] & q) {
        X[0] ^= low;  // invert the low bits of the first axis
      } else {        // exchange the low bits of the first axis and axis i
        const uint32_t t = (X[0] ^ X[i]) & low;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  X[1] ^= X[0];  // Gray code
  X[2] ^= X[1];
  uint32_t flip = 0;
  for (uint32_t q = top; q > 1; q >>= 1)
    if (X[2] & q) flip ^= q - 1;
  for (int i = 0; i < 3; ++i) X[i] ^= flip;
  uint64_t h = 0;
  for (int b = bits - 1; b >= 0; --b)
    for (int i = 0; i < 3; ++i) h = (h << 1) | ((X[i] >> b) & 1u);
  return h;
}

namespace {

std::vector<int64_t> brio_hilbert(const float* xyz, int64_t n, uint64_t seed) {
  constexpr int kBits = 16;
  std::vector<int64_t> perm = random_permutation(n, seed);
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) lo[d] = hi[d] = n ? xyz[d] : 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], (double)xyz[3 * i + d]);
      hi[d] = std::max(hi[d], (double)xyz[3 * i + d]);
    }
  double span = 0.0;
  for (int d = 0; d < 3; ++d) span = std::max(span, hi[d] - lo[d]);
  const double scale = span > 0 ? ((1u << kBits) - 1) / span : 0.0;
  auto key = [&](int64_t i) {
    uint32_t c[3];
    for (int d = 0; d < 3; ++d)
      c[d] = (uint32_t)std::min<double>((xyz[3 * i + d] - lo[d]) * scale, (1u << kBits) - 1);
    return hilbert_index3(c[0], c[1], c[2], kBits);
  };
  // rounds: [0, n>>R), [n>>R, n>>(R-1)), ..., [n>>1, n), the first at most 64 points
  std::vector<int64_t> cuts = {n};
  while (cuts.back() > 64) cuts.push_back(cuts.back() / 2);
  cuts.push_back(0);
  std::reverse(cuts.begin(), cuts.end());
  std::vector<std::pair<uint64_t, int64_t>> buf;
  for (size_t r = 0; r + 1 < cuts.size(); ++r) {
    buf.clear();
    for (int64_t t = cuts[r]; t < cuts[r + 1]; ++t) buf.push_back({key(perm[t]), perm[t]});
    std::sort(buf.begin(), buf.end());
    for (size_t t = 0; t < buf.size(); ++t) perm[cuts[r] + (int64_t)t] = buf[t].second;
  }
  return perm;
}

// Farthest-point order with a uniform grid: after a point is taken, only
// points closer to it than the current largest remaining distance can
// change, so only the grid cells within that radius are visited. A lazy
// max-heap of (distance, -index) finds the next point.
std::vector<int64_t> farthest_point(const float* xyz, int64_t n) {
  std::vector<int64_t> out;
  out.reserve((size_t)n);
  if (n == 0) return out;
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) lo[d] = hi[d] = xyz[d];
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], (double)xyz[3 * i + d]);
      hi[d] = std::max(hi[d], (double)xyz[3 * i + d]);
    }
  double span = 0.0;
  for (int d = 0; d < 3; ++d) span = std::max(span, hi[d] - lo[d]);
  const int64_t g = std::max<int64_t>(1, std::min<int64_t>(512, (int64_t)std::cbrt(n / 2.0)));
  const double cell = span > 0 ? span / g * (1 + 1e-9) : 1.0;
  auto cidx = [&](double v, int d) {
    return std::min<int64_t>(g - 1, std::max<int64_t>(0, (int64_t)((v - lo[d]) / cell)));
  };
  std::vector<int64_t> start((size_t)(g * g * g + 1), 0), pts((size_t)n);
  std::vector<int64_t> cid((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    cid[i] = (cidx(xyz[3 * i], 0) * g + cidx(xyz[3 * i + 1], 1)) * g + cidx(xyz[3 * i + 2], 2);
    start[cid[i] + 1]++;
  }
  for (size_t c = 1; c < start.size(); ++c) start[c] += start[c - 1];
  {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < n; ++i) pts[fill[cid[i]]++] = i;
  }
  std::vector<double> mind((size_t)n, INFINITY);
  std::vector<uint8_t> taken((size_t)n, 0);
  std::priority_queue<std::pair<double, int64_t>> heap;  // (distance, -index)
  int64_t next = 0;
  double radius = INFINITY;
  for (int64_t step = 0; step < n; ++step) {
    taken[next] = 1;
    mind[next] = 0.0;
    out.push_back(next);
    const double px = xyz[3 * next], py = xyz[3 * next + 1], pz = xyz[3 * next + 2];
    // cells within `radius` of the new point (all of them while it is infinite)
    int64_t c0[3], c1[3];
    const double p[3] = {px, py, pz};
    for (int d = 0; d < 3; ++d) {
      if (std::isinf(radius)) {
        c0[d] = 0;
        c1[d] = g - 1;
      } else {
        c0[d] = cidx(p[d] - radius, d);
        c1[d] = cidx(p[d] + radius, d);
      }
    }
    for (int64_t a = c0[0]; a <= c1[0]; ++a)
      for (int64_t b = c0[1]; b <= c1[1]; ++b)
        for (int64_t c = c0[2]; c <= c1[2]; ++c) {
          const int64_t cc = (a * g + b) * g + c;
          for (int64_t t = start[cc]; t < start[cc + 1]; ++t) {
            const int64_t i = pts[t];
            if (taken[i]) continue;
            const double dx = xyz[3 * i] - px, dy = xyz[3 * i + 1] - py, dz = xyz[3 * i + 2] - pz;
            const double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < mind[i]) {
              mind[i] = d2;
              heap.push({d2, -i});
            }
          }
        }
    // the next point: the largest current distance (stale heap entries skipped)
    next = -1;
    while (!heap.empty()) {
      const auto top = heap.top();
      const int64_t i = -top.second;
      if (taken[i] || top.first != mind[i]) {
        heap.pop();
        continue;
      }
      next = i;
      break;
    }
    if (next < 0) break;
    radius = std::sqrt(mind[next]) * (1 + 1e-12);
  }
  return out;
}

}  // namespace

}  // namespace mknn

using namespace mknn;

extern "C" {

mknn_status mknn_insertion_order(const float* xyz, int64_t n, int32_t kind, uint64_t seed,
                                 int64_t* order_out) {
  if (n < 0 || (n > 0 && (!xyz || !order_out))) return ofail(MKNN_EINVAL, "bad arguments");
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(xyz[i])) return ofail(MKNN_EINVAL, "non-finite coordinate");
  std::vector<int64_t> o;
  try {
    switch (kind) {
      case MKNN_ORDER_RANDOM: o = random_permutation(n, seed); break;
      case MKNN_ORDER_BRIO_HILBERT: o = brio_hilbert(xyz, n, seed); break;
      case MKNN_ORDER_FARTHEST_POINT: o = farthest_point(xyz, n); break;
      default: return ofail(MKNN_EINVAL, "unknown order kind");
    }
  } catch (const std::bad_alloc&) {
    return ofail(MKNN_ENOMEM, "host allocation failed");
  }
  if ((int64_t)o.size() != n) return ofail(MKNN_EINVAL, "order incomplete");
  std::copy(o.begin(), o.end(), order_out);
  return MKNN_OK;
}

uint64_t mknn_hilbert_index3(uint32_t x, uint32_t y, uint32_t z, int32_t bits) {
  if (bits < 1 || bits > 21) return 0;
  return hilbert_index3(x, y, z, bits);
}

}  // extern "C"
