// Lock-free union-find on a device array of parent indices.
//
// Invariant: parent[x] <= x, and every root is the minimum of its set, because a union
// only ever hooks the larger of two roots below the smaller one (atomicCAS on the larger
// root's self-loop). Finds halve paths with plain stores; a stale value read by another
// thread is still an ancestor, so halving never breaks a set. Parent loads bypass L1
// (ld.global.cg) so hooks made on other SMs are seen through L2.
#pragma once

namespace vr {

__device__ __forceinline__ int uf_load(const int *parent, int x) { return __ldcg(parent + x); }

__device__ __forceinline__ int uf_find(int *parent, int x) {
  while (true) {
    int p = uf_load(parent, x);
    if (p == x) return x;
    int gp = uf_load(parent, p);
    if (gp == p) return p;
    parent[x] = gp;
    x = gp;
  }
}

__device__ __forceinline__ void uf_unite(int *parent, int a, int b) {
  while (true) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a > b) {
      int t = a;
      a = b;
      b = t;
    }
    // hook root b (larger) below a
    int old = atomicCAS(parent + b, b, a);
    if (old == b) return;
    b = old;
  }
}

}  // namespace vr
