// Flood-fill refinement order (Sec. 4.2), host code.
//
// The greedy refinement is order dependent; the paper refines the least
// covered interesting cell first and then spreads to its neighbours through
// a priority queue.  Fixed here: the priority of a cell is its covered
// sub-point count (lowest first, ties to the lower list index); the
// neighbours of a cell are the listed cells that share a face, an edge or a
// corner with it; when the queue runs dry the least covered cell not yet
// emitted starts the next flood.  Every cell enters the queue once.
#include <algorithm>
#include <cstdint>
#include <queue>
#include <unordered_map>
#include <vector>

#include "gfs.h"

namespace {

struct Key {
  uint32_t count;
  int64_t index;
  bool operator>(const Key& o) const { return count != o.count ? count > o.count : index > o.index; }
};

// cells are at most 2^20 apart per axis (checked by the caller), so three
// biased 21-bit fields identify a cell
inline uint64_t pack(int64_t i, int64_t j, int64_t k) {
  const int64_t b = int64_t(1) << 20;
  return (uint64_t(i + b) << 42) | (uint64_t(j + b) << 21) | uint64_t(k + b);
}

}  // namespace

extern "C" int gfs_flood_order(const int32_t* cells_host, const uint32_t* counts_host, int64_t ncells,
                               int64_t* order_out_host) {
  if (ncells < 0 || (ncells > 0 && (!cells_host || !counts_host || !order_out_host))) return GFS_ERR_ARG;
  const int64_t lim = (int64_t(1) << 20) - 2;
  for (int64_t c = 0; c < 3 * ncells; ++c)
    if (cells_host[c] < -lim || cells_host[c] > lim) return GFS_ERR_TOO_LARGE;
  std::unordered_map<uint64_t, int64_t> where;
  where.reserve(size_t(ncells) * 2);
  for (int64_t c = 0; c < ncells; ++c) {
    const uint64_t key = pack(cells_host[3 * c], cells_host[3 * c + 1], cells_host[3 * c + 2]);
    if (!where.emplace(key, c).second) return GFS_ERR_ARG;  // a cell listed twice
  }
  std::vector<int64_t> seeds(static_cast<size_t>(ncells));
  for (int64_t c = 0; c < ncells; ++c) seeds[c] = c;
  std::sort(seeds.begin(), seeds.end(), [&](int64_t a, int64_t b) {
    return counts_host[a] != counts_host[b] ? counts_host[a] < counts_host[b] : a < b;
  });
  std::vector<char> queued(static_cast<size_t>(ncells), 0);
  std::priority_queue<Key, std::vector<Key>, std::greater<Key>> heap;
  int64_t emitted = 0;
  size_t next_seed = 0;
  while (emitted < ncells) {
    if (heap.empty()) {
      while (queued[seeds[next_seed]]) ++next_seed;
      const int64_t s = seeds[next_seed];
      queued[s] = 1;
      heap.push(Key{counts_host[s], s});
    }
    const int64_t c = heap.top().index;
    heap.pop();
    order_out_host[emitted++] = c;
    const int64_t ci = cells_host[3 * c], cj = cells_host[3 * c + 1], ck = cells_host[3 * c + 2];
    for (int di = -1; di <= 1; ++di)
      for (int dj = -1; dj <= 1; ++dj)
        for (int dk = -1; dk <= 1; ++dk) {
          if (!di && !dj && !dk) continue;
          const auto it = where.find(pack(ci + di, cj + dj, ck + dk));
          if (it == where.end() || queued[it->second]) continue;
          queued[it->second] = 1;
          heap.push(Key{counts_host[it->second], it->second});
        }
  }
  return GFS_OK;
}
