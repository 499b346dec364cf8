// Octree cell walk on the device (grid kind 1).  A packet in a leaf carries
// the leaf's level, its integer coordinates at that level and the local
// position xi in [0, 1]^3 in units of the leaf size, exactly like a Cartesian
// cell.  Crossing a face looks up the node across it (same level or coarser,
// precomputed per leaf face) and descends to the leaf that contains the face
// point.  Points on a split plane go to the side the direction enters (the
// half-open rule of the Cartesian walk; a zero direction component counts as
// entering the upper side).
#pragma once
#include "cellpos.cuh"
#include "internal.h"

namespace colt {

// 2^-n for 0 <= n < 127 (FP32) / 1023 (FP64), exact
template <typename R>
__device__ __forceinline__ R pow2neg(int n);
template <>
__device__ __forceinline__ float pow2neg<float>(int n) { return __int_as_float((127 - n) << 23); }
template <>
__device__ __forceinline__ double pow2neg<double>(int n) {
  return __longlong_as_double((long long)(1023 - n) << 52);
}

// Leaf of the octree containing the local point f (in units of node v's size,
// v of level *lvl with integer coordinates ci), descending from v.  f, ci and
// *lvl are updated to the leaf's; returns the leaf index.
template <typename R>
__device__ __forceinline__ int64_t oct_descend(const GridDev& G, uint32_t v, const R k[3], CellPos<R> f[3],
                                               int ci[3], int* lvl) {
  int32_t ch;
  while ((ch = __ldg(G.node + v)) >= 0) {
    int cidx = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int up = f[a].descend(k[a] >= R(0));
      ci[a] = 2 * ci[a] + up;
      cidx |= up << a;
    }
    v = (uint32_t)ch + (uint32_t)cidx;
    ++*lvl;
  }
  return -1 - (int64_t)ch;
}

// The neighbour-table entry of leaf `cell`'s face on axis ax towards sgn.
__device__ __forceinline__ uint32_t oct_face_entry(const GridDev& G, int64_t cell, int ax, int sgn) {
  return __ldg(G.nbr + 6 * cell + 2 * ax + (sgn > 0 ? 0 : 1));
}

// Cross a face whose neighbour-table entry nb the caller has loaded (a walk
// loads the next face's entry together with the leaf's record, so that the
// two loads overlap).  The packet lies on that face of the current leaf.
// Returns the new leaf, or -1 when the face is the box boundary; ci, *lvl and
// xi become the new leaf's.
template <typename R>
__device__ __forceinline__ int64_t oct_cross_entry(const GridDev& G, uint32_t nb, int ax, int sgn, const R k[3],
                                                   int ci[3], int* lvl, CellPos<R> xi[3]) {
  if (nb == kNoNbr) return -1;
  const int ln = (int)(nb >> 27);
  const int d = *lvl - ln;
  const R sc = pow2neg<R>(d);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int adj = ci[a] + (a == ax ? sgn : 0);
    const int top = adj >> d;                   // the node's coordinate at level ln
    if (a == ax) xi[a].set(sgn > 0 ? R(0) : R(1));
    else xi[a].shift_scale(adj - (top << d), sc);
    ci[a] = top;
  }
  *lvl = ln;
  if (nb & kLeafFlag) return (int64_t)(nb & kNodeMask);   // a leaf of that level: no descent
  return oct_descend<R>(G, nb & kNodeMask, k, xi, ci, lvl);
}

// Cross the face of leaf `cell` on axis ax towards sgn (oct_cross_entry with
// the entry loaded here).
template <typename R>
__device__ __forceinline__ int64_t oct_cross(const GridDev& G, int64_t cell, int ax, int sgn, const R k[3],
                                             int ci[3], int* lvl, CellPos<R> xi[3]) {
  return oct_cross_entry<R>(G, oct_face_entry(G, cell, ax, sgn), ax, sgn, k, ci, lvl, xi);
}

}  // namespace colt
