// Device helpers shared by the stencil and V-cycle translation units: the
// boundary test, one row of the Helmholtz / CSLP operator and bilinear
// interpolation, for any storage type of the vector they read.
#pragma once

#include <cuda_bf16.h>

#include "hz_common.cuh"

namespace hz {

__device__ __forceinline__ float2 ld2(const __nv_bfloat162* p, long long i) {
  return __bfloat1622float2(p[i]);
}
__device__ __forceinline__ void st2(__nv_bfloat162* p, long long i, float2 v) {
  p[i] = __float22bfloat162_rn(v);
}

__device__ __forceinline__ bool on_bnd(int i, int j, int nx, int ny) {
  return i == 0 || j == 0 || i == nx - 1 || j == ny - 1;
}

// Row (i, j) of M = -Lap - (sre + i sim) k^2 with the boundary rules of
// helm_point below: centre and the four neighbour weights (0 where the
// neighbour is outside the grid or a Dirichlet boundary node).  k2 is the
// node's squared wavenumber, loaded by the caller (so that the load can be
// issued ahead of its use).
template <class T>
__device__ __forceinline__ void helm_row(const LevelDev& L, int bc, T sre, T sim, int i,
                                         int j, T k2, C<T>& cen, T& cw, T& ce, T& cs,
                                         T& cn) {
  const int nx = L.nx, ny = L.ny;
  const T ih2 = ih2_of<T>(L);
  cen = mkc(T(4) * ih2 - sre * k2, -sim * k2);
  cw = -ih2;
  ce = -ih2;
  cs = -ih2;
  cn = -ih2;
  if (bc == BC_SOMMERFELD) {
    const bool x0 = i == 0, x1 = i == nx - 1, y0 = j == 0, y1 = j == ny - 1;
    const int ns = int(x0) + int(x1) + int(y0) + int(y1);
    if (ns) {
      cen.y -= T(ns) * tih_of<T>(L) * sqrt(k2);
      if (x0) { cw = T(0); ce = T(2) * ce; }
      if (x1) { ce = T(0); cw = T(2) * cw; }
      if (y0) { cs = T(0); cn = T(2) * cn; }
      if (y1) { cn = T(0); cs = T(2) * cs; }
    }
  } else {
    if (i == 1) cw = T(0);
    if (i == nx - 2) ce = T(0);
    if (j == 1) cs = T(0);
    if (j == ny - 2) cn = T(0);
  }
}

// (M x)(i, j) for an unknown node (i, j): centre 4/h^2 - s k^2, Sommerfeld
// sides add -2 i k / h each, remove the outward neighbour and double the
// opposite one (ghost elimination); Dirichlet rows drop couplings to the
// (fixed zero) boundary nodes.  x is stored as SX, the arithmetic is C<T>.
template <class T, class SX>
__device__ __forceinline__ C<T> helm_point(const LevelDev& L, int bc, T sre,
                                           T sim, const SX* __restrict__ x,
                                           int i, int j) {
  const int nx = L.nx, ny = L.ny;
  const long long id = (long long)j * nx + i;
  const T ih2 = ih2_of<T>(L);
  const T k2 = k2_of<T>(L)[id];
  C<T> cen = mkc(T(4) * ih2 - sre * k2, -sim * k2);
  T cw = -ih2, ce = -ih2, cs = -ih2, cn = -ih2;
  if (bc == BC_SOMMERFELD) {
    const bool x0 = i == 0, x1 = i == nx - 1, y0 = j == 0, y1 = j == ny - 1;
    const int ns = int(x0) + int(x1) + int(y0) + int(y1);
    if (ns) {
      cen.y -= T(ns) * tih_of<T>(L) * sqrt(k2);
      if (x0) { cw = T(0); ce = T(2) * ce; }
      if (x1) { ce = T(0); cw = T(2) * cw; }
      if (y0) { cs = T(0); cn = T(2) * cn; }
      if (y1) { cn = T(0); cs = T(2) * cs; }
    }
  } else {
    if (i == 1) cw = T(0);
    if (i == nx - 2) ce = T(0);
    if (j == 1) cs = T(0);
    if (j == ny - 2) cn = T(0);
  }
  C<T> acc = cmul(cen, ld2(x, id));
  if (cw != T(0)) acc = rfma(cw, ld2(x, id - 1), acc);
  if (ce != T(0)) acc = rfma(ce, ld2(x, id + 1), acc);
  if (cs != T(0)) acc = rfma(cs, ld2(x, id - nx), acc);
  if (cn != T(0)) acc = rfma(cn, ld2(x, id + nx), acc);
  return acc;
}

// bilinear interpolation of the coarse vector xc (stored as SC) at fine
// node (i, j)
template <class T, class SC>
__device__ __forceinline__ C<T> interp_bilinear(const LevelDev& Lc,
                                                const SC* __restrict__ xc,
                                                int i, int j) {
  const int I0 = i >> 1, J0 = j >> 1;
  const bool ox = i & 1, oy = j & 1;
  const long long b0 = (long long)J0 * Lc.nx + I0;
  if (!ox && !oy) return ld2(xc, b0);
  if (ox && !oy) return T(0.5) * (ld2(xc, b0) + ld2(xc, b0 + 1));
  if (!ox && oy) return T(0.5) * (ld2(xc, b0) + ld2(xc, b0 + Lc.nx));
  return T(0.25) * ((ld2(xc, b0) + ld2(xc, b0 + 1)) +
                    (ld2(xc, b0 + Lc.nx) + ld2(xc, b0 + Lc.nx + 1)));
}

// Asynchronous global -> shared copies of one element (cp.async, completing
// per thread in commit groups; the data is visible to other threads after
// cp.async.wait_group and a block barrier).  The element size (4, 8 or 16
// bytes) is also the alignment both addresses have.
template <int BYTES>
__device__ __forceinline__ void cp_async_el(void* smem, const void* gmem) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}
// zero of a storage type (for tile entries outside the grid)
template <class S> __device__ __forceinline__ S szero() {
  S v;
  memset(&v, 0, sizeof(S));
  return v;
}

}  // namespace hz
