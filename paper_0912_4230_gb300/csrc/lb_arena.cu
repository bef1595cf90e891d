// Packed lattice arena: sub-allocation of one device region for the
// lattices of a serving loop (see lb_arena_* in lb.h).
#include <cuda_runtime.h>

#include <cstdint>
#include <iterator>
#include <map>
#include <mutex>
#include <new>

#include "../../include/lb.h"

struct lb_arena {
  char *base = nullptr;
  size_t bytes = 0;
  bool owned = false;                  // allocated here with cudaMalloc
  std::map<size_t, size_t> free_list;  // offset -> length, address order
  std::map<size_t, size_t> live;       // offset -> length of handed-out blocks
  size_t used = 0, peak = 0;
  mutable std::mutex mu;
};

namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

void *arena_alloc_fn(size_t bytes, void *user) {
  return lb_arena_alloc(static_cast<lb_arena *>(user), bytes);
}
void arena_release_fn(void *ptr, void *user) { lb_arena_free(static_cast<lb_arena *>(user), ptr); }

}  // namespace

extern "C" {

int lb_arena_create(void *base, size_t bytes, lb_arena **out) {
  if (!out) return LB_EINVAL;
  *out = nullptr;
  if (bytes < kAlign) return LB_EINVAL;
  if (base && reinterpret_cast<uintptr_t>(base) % kAlign) return LB_EINVAL;
  lb_arena *a = new (std::nothrow) lb_arena;
  if (!a) return LB_ENOMEM;
  a->bytes = bytes / kAlign * kAlign;
  if (base) {
    a->base = static_cast<char *>(base);
  } else {
    void *p = nullptr;
    if (cudaMalloc(&p, a->bytes) != cudaSuccess) {
      cudaGetLastError();
      delete a;
      return LB_ENOMEM;
    }
    a->base = static_cast<char *>(p);
    a->owned = true;
  }
  a->free_list[0] = a->bytes;
  *out = a;
  return LB_OK;
}

void lb_arena_destroy(lb_arena *a) {
  if (!a) return;
  if (a->owned) cudaFree(a->base);
  delete a;
}

int lb_arena_use(lb_arena *a) {
  return a ? lb_set_allocator(arena_alloc_fn, arena_release_fn, a)
           : lb_set_allocator(nullptr, nullptr, nullptr);
}

void *lb_arena_alloc(lb_arena *a, size_t bytes) {
  // larger than the region: nothing fits (and rounding it up could wrap to 0)
  if (!a || bytes == 0 || bytes > a->bytes) return nullptr;
  const size_t need = round_up(bytes);
  std::lock_guard<std::mutex> lock(a->mu);
  for (auto it = a->free_list.begin(); it != a->free_list.end(); ++it) {
    if (it->second < need) continue;
    const size_t off = it->first, len = it->second;
    a->free_list.erase(it);
    if (len > need) a->free_list[off + need] = len - need;
    a->live[off] = need;
    a->used += need;
    if (a->used > a->peak) a->peak = a->used;
    return a->base + off;
  }
  return nullptr;
}

void lb_arena_free(lb_arena *a, void *ptr) {
  if (!a || !ptr) return;
  const uintptr_t p = reinterpret_cast<uintptr_t>(ptr), b = reinterpret_cast<uintptr_t>(a->base);
  if (p < b || p - b >= a->bytes) return;  // outside the region
  const size_t off = size_t(p - b);
  std::lock_guard<std::mutex> lock(a->mu);
  auto lv = a->live.find(off);
  if (lv == a->live.end()) return;  // not a block of this arena
  size_t start = off, len = lv->second;
  a->live.erase(lv);
  a->used -= len;
  // merge with the free neighbours on either side
  auto next = a->free_list.lower_bound(start);
  if (next != a->free_list.end() && next->first == start + len) {
    len += next->second;
    next = a->free_list.erase(next);
  }
  if (next != a->free_list.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == start) {
      start = prev->first;
      len += prev->second;
      a->free_list.erase(prev);
    }
  }
  a->free_list[start] = len;
}

int lb_arena_stats(const lb_arena *a, size_t *used, size_t *largest_free, size_t *peak,
                   size_t *blocks) {
  if (!a) return LB_EINVAL;
  std::lock_guard<std::mutex> lock(a->mu);
  size_t big = 0;
  for (const auto &f : a->free_list) big = f.second > big ? f.second : big;
  if (used) *used = a->used;
  if (largest_free) *largest_free = big;
  if (peak) *peak = a->peak;
  if (blocks) *blocks = a->live.size();
  return LB_OK;
}

}  // extern "C"
