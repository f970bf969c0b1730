// serve_tile.cuh -- the tiles of a serving round's work list (ServeList,
// internal.h), as the serving instantiations of the solve kernels see them.
#pragma once

#include <cstdint>

#include "internal.h"

namespace syev3 {

// One tile: its first input record, its output rows and its matrix count.
template <class T>
struct TileRef {
  const T* src;
  T* lam;
  T* U;  // null: eigenvalues only
  int cnt;
};

// Tile `tile` (< list->n_tiles) of the list.  `cur` is the caller's item
// cursor, 0 at the start: a CTA visits its tiles in increasing order, so the
// cursor only moves forward and each item is stepped over once.
template <class T>
__device__ __forceinline__ TileRef<T> serve_tile(const ServeList* list, int64_t tile, int64_t& cur) {
  const int64_t ni = list->n_items;
  while (cur + 1 < ni && list->items[cur + 1].tile_begin <= tile) ++cur;
  const ServeItem& it = list->items[cur];
  const int64_t base = (tile - it.tile_begin) * kServeTile;
  const int64_t left = it.count - base;
  TileRef<T> r;
  r.cnt = (int)(left < kServeTile ? left : kServeTile);
  r.src = static_cast<const T*>(it.A) + base * 6;
  r.lam = static_cast<T*>(it.lam) + base * 3;
  r.U = it.U ? static_cast<T*>(it.U) + base * 9 : nullptr;
  return r;
}

}  // namespace syev3
