// Host-side rules of Alg. 3 (R_block): where the channel blocks of R are
// decoupled.  Plain C++ (no CUDA), shared by the library's setup and its
// host-logic test.
#pragma once
#include <algorithm>
#include <utility>
#include <vector>

namespace wc4d {

// Alg. 3 on the host: the rows where R_block decouples.  A cut c separates
// rows < c from rows >= c; runs are the row ranges between cuts.
inline std::vector<int> rblock_cuts(const std::vector<int>& sizes, const std::vector<double>& normvec, double tol,
                                    int maxsize, int numproc, int p) {
  std::vector<int> cuts;
  int start = 0;
  for (size_t j = 0; j + 1 < sizes.size(); ++j) {
    start += sizes[j];
    if (normvec[j] < tol) cuts.push_back(start);
  }
  auto runs = [&]() {
    std::vector<std::pair<int, int>> r;
    int a = 0;
    for (int c : cuts) {
      r.push_back({a, c});
      a = c;
    }
    r.push_back({a, p});
    return r;
  };
  auto split_largest = [&]() {
    const auto r = runs();
    size_t best = 0;
    for (size_t i = 1; i < r.size(); ++i)
      if (r[i].second - r[i].first > r[best].second - r[best].first) best = i;
    const int a = r[best].first, len = r[best].second - r[best].first;
    if (len >= 2) {
      cuts.push_back(a + len / 2);
      std::sort(cuts.begin(), cuts.end());
    }
  };
  if (maxsize > 0) {
    int largest = 0;
    for (const auto& q : runs()) largest = std::max(largest, q.second - q.first);
    if (largest > maxsize) split_largest();
  }
  if (numproc > 0) {
    const auto r = runs();
    const int nr = (int)r.size();
    if (nr > numproc) {
      size_t best = 0;
      for (size_t i = 1; i + 1 < r.size(); ++i)
        if (r[i + 1].second - r[i].first < r[best + 1].second - r[best].first) best = i;
      cuts.erase(std::find(cuts.begin(), cuts.end(), r[best].second));
    } else if (nr < numproc - 2) {
      split_largest();
    }
  }
  return cuts;
}

}  // namespace wc4d
