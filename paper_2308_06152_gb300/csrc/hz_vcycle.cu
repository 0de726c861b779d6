// Kernels of the CSLP multigrid V-cycle (Sec. 3.1, Sec. 5.1): damped-Jacobi
// sweeps (w = 0.8) with the residual fused into full-weighting restriction
// (eq. weight operator), bilinear interpolation of the correction (eq.
// bilinear operator) and the dense coarsest-level solve.  Vectors of the
// level hierarchy may be stored in a narrower type than the arithmetic
// (BF16 pairs for the smoother variant); the arithmetic is C<T>.
#include <mutex>

#include "hz_common.cuh"
#include "hz_stencil_dev.cuh"

namespace hz {

namespace {

constexpr int BX = 32, BY = 8;

inline dim3 grid2d(int nx, int ny, int nrhs) {
  return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, nrhs);
}

// x = dinv .* f (one damped-Jacobi sweep from x = 0)
template <class T, class SF, class SX>
__global__ void k_jacobi0(LevelDev L, int bc, VRefE<SF> fin, SX* __restrict__ x,
                          const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || (done && done[r])) return;
  const long long n = (long long)L.nx * L.ny, id = (long long)j * L.nx + i;
  if (bc == BC_DIRICHLET && on_bnd(i, j, L.nx, L.ny)) {
    st2(x, r * n + id, czero<T>());
    return;
  }
  st2(x, r * n + id, cmul(dinv_of<T>(L)[id], ld2(fin.get(), r * n + id)));
}

// fc(I,J) = sum_{a,b in -1..1} (2-|a|)(2-|b|)/16 * (f - M x)(2I+a, 2J+b)
template <class T, class SF, class SX, class SC>
__global__ void k_resid_restrict(LevelDev Lf, LevelDev Lc, int bc, T sre, T sim,
                                 VRefE<SF> fin, const SX* __restrict__ x,
                                 SC* __restrict__ fc, const int* __restrict__ done) {
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (I >= Lc.nx || J >= Lc.ny || (done && done[r])) return;
  const long long nf = (long long)Lf.nx * Lf.ny, nc = (long long)Lc.nx * Lc.ny;
  const long long idc = (long long)J * Lc.nx + I;
  if (bc == BC_DIRICHLET && on_bnd(I, J, Lc.nx, Lc.ny)) {
    st2(fc, r * nc + idc, czero<T>());
    return;
  }
  const SF* f = fin.get() + r * nf;
  const SX* xr = x + r * nf;
  C<T> acc = czero<T>();
  for (int b = -1; b <= 1; ++b) {
    const int jf = 2 * J + b;
    if (jf < 0 || jf >= Lf.ny) continue;
    for (int a = -1; a <= 1; ++a) {
      const int ifn = 2 * I + a;
      if (ifn < 0 || ifn >= Lf.nx) continue;
      if (bc == BC_DIRICHLET && on_bnd(ifn, jf, Lf.nx, Lf.ny)) continue;
      const C<T> res = ld2(f, (long long)jf * Lf.nx + ifn) -
                       helm_point<T, SX>(Lf, bc, sre, sim, xr, ifn, jf);
      const T w = T((2 - abs(a)) * (2 - abs(b))) * T(0.0625);
      acc = rfma(w, res, acc);
    }
  }
  st2(fc, r * nc + idc, acc);
}

// x += P_bilinear xc
template <class T, class SC, class SX>
__global__ void k_prolong_add(LevelDev Lf, LevelDev Lc, int bc,
                              const SC* __restrict__ xc, SX* __restrict__ x,
                              const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= Lf.nx || j >= Lf.ny || (done && done[r])) return;
  if (bc == BC_DIRICHLET && on_bnd(i, j, Lf.nx, Lf.ny)) return;
  const long long nf = (long long)Lf.nx * Lf.ny, nc = (long long)Lc.nx * Lc.ny;
  const long long id = (long long)j * Lf.nx + i;
  st2(x, r * nf + id, ld2(x, r * nf + id) + interp_bilinear<T, SC>(Lc, xc + r * nc, i, j));
}

// xo = x + dinv .* (f - M x)
template <class T, class SF, class SX, class SO>
__global__ void k_smooth(LevelDev L, int bc, T sre, T sim, VRefE<SF> fin,
                         const SX* __restrict__ x, SO* __restrict__ xo,
                         const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || (done && done[r])) return;
  const long long n = (long long)L.nx * L.ny, id = (long long)j * L.nx + i;
  if (bc == BC_DIRICHLET && on_bnd(i, j, L.nx, L.ny)) {
    st2(xo, r * n + id, czero<T>());
    return;
  }
  const SX* xr = x + r * n;
  const C<T> res = ld2(fin.get(), r * n + id) - helm_point<T, SX>(L, bc, sre, sim, xr, i, j);
  st2(xo, r * n + id, cfma(dinv_of<T>(L)[id], res, ld2(xr, id)));
}

// Fused pre-smoothing, residual and restriction for one BX x BY tile of
// coarse nodes: x = dinv .* f on the fine nodes [2I0-2, 2I0+2BX] (+1) held
// in shared memory (the tile's own fine nodes are also written out), then
// f - M x on [2I0-1, 2I0+2BX-1] and its full weighting.  x is computed
// from f where it is needed instead of being read back, so the pair reads
// f once and writes x and the coarse right-hand side once.  Every global
// load a thread needs (D^-1 and f of its x nodes, f and k^2 of its
// residual nodes) is issued up front into registers, so each thread has
// all its loads in flight at once instead of one per loop trip, and the
// residual's operands arrive while the x tile is being built.
template <class T, class SF, class SX, class SC>
__global__ void __launch_bounds__(BX * BY)
k_pre_restrict(LevelDev Lf, LevelDev Lc, int bc, T sre, T sim, VRefE<SF> fin,
               SX* __restrict__ x, SC* __restrict__ fc, const int* __restrict__ done) {
  constexpr int XW = 2 * BX + 3, XH = 2 * BY + 3, RW = 2 * BX + 1, RH = 2 * BY + 1;
  constexpr int NT = BX * BY;
  constexpr int N1 = (XH * XW + NT - 1) / NT, N2 = (RH * RW + NT - 1) / NT;
  __shared__ C<T> xs[XH * XW];
  __shared__ C<T> rsd[RH * RW];
  const int r = blockIdx.z;
  if (done && done[r]) return;
  const int I0 = blockIdx.x * BX, J0 = blockIdx.y * BY;
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int nfx = Lf.nx, nfy = Lf.ny;
  const long long nf = (long long)nfx * nfy, nc = (long long)Lc.nx * Lc.ny;
  const SF* f = fin.get() + r * nf;
  SX* xr = x + r * nf;
  const C<T>* dinv = dinv_of<T>(Lf);
  const T* k2f = k2_of<T>(Lf);
  // operands of the x tile (zero outside the grid and on Dirichlet
  // boundary nodes, where x = 0)
  C<T> dv[N1], fv[N1];
#pragma unroll
  for (int u = 0; u < N1; ++u) {
    const int q = tid + u * NT;
    const int gi = 2 * I0 - 2 + q % XW, gj = 2 * J0 - 2 + q / XW;
    dv[u] = czero<T>();
    fv[u] = czero<T>();
    if (q < XH * XW && gi >= 0 && gi < nfx && gj >= 0 && gj < nfy &&
        !(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy))) {
      const long long id = (long long)gj * nfx + gi;
      dv[u] = dinv[id];
      fv[u] = ld2(f, id);
    }
  }
  // operands of the residual nodes
  C<T> f2[N2];
  T k2v[N2];
#pragma unroll
  for (int u = 0; u < N2; ++u) {
    const int q = tid + u * NT;
    const int gi = 2 * I0 - 1 + q % RW, gj = 2 * J0 - 1 + q / RW;
    f2[u] = czero<T>();
    k2v[u] = T(0);
    if (q < RH * RW && gi >= 0 && gi < nfx && gj >= 0 && gj < nfy &&
        !(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy))) {
      const long long id = (long long)gj * nfx + gi;
      f2[u] = ld2(f, id);
      k2v[u] = k2f[id];
    }
  }
#pragma unroll
  for (int u = 0; u < N1; ++u) {
    const int q = tid + u * NT;
    if (q < XH * XW) {
      const int gi = 2 * I0 - 2 + q % XW, gj = 2 * J0 - 2 + q / XW;
      const C<T> v = cmul(dv[u], fv[u]);
      if (gi >= 2 * I0 && gi < 2 * I0 + 2 * BX && gi < nfx && gj >= 2 * J0 &&
          gj < 2 * J0 + 2 * BY && gj < nfy)
        st2(xr, (long long)gj * nfx + gi, v);
      xs[q] = v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < N2; ++u) {
    const int q = tid + u * NT;
    if (q < RH * RW) {
      const int ri = q % RW, rj = q / RW;
      const int gi = 2 * I0 - 1 + ri, gj = 2 * J0 - 1 + rj;
      C<T> v = czero<T>();
      if (gi >= 0 && gi < nfx && gj >= 0 && gj < nfy &&
          !(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy))) {
        C<T> cen;
        T cw, ce, cs, cn;
        helm_row<T>(Lf, bc, sre, sim, gi, gj, k2v[u], cen, cw, ce, cs, cn);
        const int c = (rj + 1) * XW + (ri + 1);
        C<T> acc = cmul(cen, xs[c]);
        if (cw != T(0)) acc = rfma(cw, xs[c - 1], acc);
        if (ce != T(0)) acc = rfma(ce, xs[c + 1], acc);
        if (cs != T(0)) acc = rfma(cs, xs[c - XW], acc);
        if (cn != T(0)) acc = rfma(cn, xs[c + XW], acc);
        v = f2[u] - acc;
      }
      rsd[q] = v;
    }
  }
  __syncthreads();
  const int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
  if (I >= Lc.nx || J >= Lc.ny) return;
  C<T> acc = czero<T>();
  if (!(bc == BC_DIRICHLET && on_bnd(I, J, Lc.nx, Lc.ny))) {
    for (int b = -1; b <= 1; ++b)
      for (int a = -1; a <= 1; ++a) {
        const T w = T((2 - abs(a)) * (2 - abs(b))) * T(0.0625);
        acc = rfma(w, rsd[(2 * threadIdx.y + 1 + b) * RW + 2 * threadIdx.x + 1 + a], acc);
      }
  }
  st2(fc, r * nc + (long long)J * Lc.nx + I, acc);
}

// Fused coarse-grid correction and post-smoothing for one BX x BY tile of
// fine nodes: x' = x + P xc on the tile and its 1-node halo in shared
// memory, then xo = x' + dinv .* (f - M x').  x' is never stored.  The
// thread's own f, D^-1 and k^2 are loaded before the tile is built, so
// they arrive while the x' loads are in flight.
template <class T, class SC, class SX, class SF, class SO>
__global__ void __launch_bounds__(BX * BY)
k_prolong_smooth(LevelDev Lf, LevelDev Lc, int bc, T sre, T sim,
                 const SC* __restrict__ xc, const SX* __restrict__ x, VRefE<SF> fin,
                 SO* __restrict__ xo, const int* __restrict__ done) {
  constexpr int PW = BX + 2, PH = BY + 2, NT = BX * BY;
  constexpr int N1 = (PH * PW + NT - 1) / NT;
  __shared__ C<T> xp[PH * PW];
  const int r = blockIdx.z;
  if (done && done[r]) return;
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int nfx = Lf.nx, nfy = Lf.ny;
  const long long nf = (long long)nfx * nfy, nc = (long long)Lc.nx * Lc.ny;
  const SX* xr = x + r * nf;
  const SC* xcr = xc + r * nc;
  const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
  const bool mine = i < nfx && j < nfy;
  const long long id = (long long)j * nfx + i;
  C<T> fown = czero<T>(), down = czero<T>();
  T k2own = T(0);
  if (mine) {
    fown = ld2(fin.get(), r * nf + id);
    down = dinv_of<T>(Lf)[id];
    k2own = k2_of<T>(Lf)[id];
  }
  C<T> xv[N1];
#pragma unroll
  for (int u = 0; u < N1; ++u) {
    const int q = tid + u * NT;
    const int gi = i0 - 1 + q % PW, gj = j0 - 1 + q / PW;
    xv[u] = czero<T>();
    if (q < PH * PW && gi >= 0 && gi < nfx && gj >= 0 && gj < nfy) {
      xv[u] = ld2(xr, (long long)gj * nfx + gi);
      if (!(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy)))
        xv[u] = xv[u] + interp_bilinear<T, SC>(Lc, xcr, gi, gj);
    }
  }
#pragma unroll
  for (int u = 0; u < N1; ++u) {
    const int q = tid + u * NT;
    if (q < PH * PW) xp[q] = xv[u];
  }
  __syncthreads();
  if (!mine) return;
  if (bc == BC_DIRICHLET && on_bnd(i, j, nfx, nfy)) {
    st2(xo, r * nf + id, czero<T>());
    return;
  }
  C<T> cen;
  T cw, ce, cs, cn;
  helm_row<T>(Lf, bc, sre, sim, i, j, k2own, cen, cw, ce, cs, cn);
  const int c = (threadIdx.y + 1) * PW + (threadIdx.x + 1);
  C<T> acc = cmul(cen, xp[c]);
  if (cw != T(0)) acc = rfma(cw, xp[c - 1], acc);
  if (ce != T(0)) acc = rfma(ce, xp[c + 1], acc);
  if (cs != T(0)) acc = rfma(cs, xp[c - PW], acc);
  if (cn != T(0)) acc = rfma(cn, xp[c + PW], acc);
  const C<T> res = fown - acc;
  st2(xo, r * nf + id, cfma(down, res, xp[c]));
}

// ---------------------------------------------------------------------------
// Multi-RHS staged variants of the two fused kernels.  One block keeps its
// tile's per-node constants (D^-1, neighbour weights, smem offsets) in
// registers and walks over a group of right-hand sides; each right-hand
// side's input tile (with its halo) is copied into a ring of NS
// shared-memory stages by cp.async, NS-1 right-hand sides ahead of the one
// being computed.  The arithmetic uses D^-1 = w / diag(M) to drop the
// diagonal of M: with x = D^-1 f, (M x)_c = w f_c + sum_nb m_nb x_nb, so
//   residual   f - M x          = (1 - w) f_c - sum_nb m_nb x_nb,
//   smoothing  x + D^-1 (f - M x) = (1 - w) x_c + D^-1_c (f_c - sum_nb m_nb x_nb),
// the same quantities as the kernels above (to rounding) without k^2 or
// the complex diagonal.  The off-diagonal m_nb is -1/h^2 times 1 inside the
// grid, 2 toward the interior at a Sommerfeld side (ghost elimination), 0
// outside the grid or toward a Dirichlet boundary node; tiles whose halo
// stays off the boundary take a path without those tests.

// RHS of [r0, r1) not yet done, listed in act[] by warp 0; returns the count
// to every thread.
__device__ __forceinline__ int list_active(const int* __restrict__ done, int r0, int r1,
                                           int* act, int* cnt_s) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid < 32) {
    int cnt = 0;
    for (int base = r0; base < r1; base += 32) {
      const int r = base + tid;
      const bool a = r < r1 && !(done && done[r]);
      const unsigned m = __ballot_sync(0xffffffffu, a);
      if (a) act[cnt + __popc(m & ((1u << tid) - 1u))] = r;
      cnt += __popc(m);
    }
    if (tid == 0) *cnt_s = cnt;
  }
  __syncthreads();
  return *cnt_s;
}

__host__ __device__ constexpr int align16(int b) { return (b + 15) & ~15; }

// Off-diagonal weights of row (i, j) of M (an unknown node) as multiples of
// -1/h^2, two bits each: west, east, south, north (see helm_row).
__device__ __forceinline__ unsigned nb_code(int bc, int i, int j, int nx, int ny) {
  unsigned w = 1, e = 1, so = 1, no = 1;
  if (bc == BC_SOMMERFELD) {
    if (i == 0) { w = 0; e = 2; }
    if (i == nx - 1) { e = 0; w = 2; }
    if (j == 0) { so = 0; no = 2; }
    if (j == ny - 1) { no = 0; so = 2; }
  } else {
    if (i == 1) w = 0;
    if (i == nx - 2) e = 0;
    if (j == 1) so = 0;
    if (j == ny - 2) no = 0;
  }
  return w | (e << 2) | (so << 4) | (no << 6);
}
// -sum_nb m_nb x_nb / (1/h^2) = sum of the neighbours with their weights
template <class T, bool INTERIOR>
__device__ __forceinline__ C<T> nb_sum(const C<T>* xs, int c, int row, unsigned code) {
  const C<T> xw = xs[c - 1], xe = xs[c + 1], xso = xs[c - row], xno = xs[c + row];
  if (INTERIOR) return (xw + xe) + (xso + xno);
  C<T> a = T(code & 3u) * xw;
  a = rfma(T((code >> 2) & 3u), xe, a);
  a = rfma(T((code >> 4) & 3u), xso, a);
  return rfma(T((code >> 6) & 3u), xno, a);
}

// Two adjacent values p[0], p[1] of a staged or shared array as one vector
// load (p aligned to twice the element size) or store.
template <class S>
__device__ __forceinline__ void ld_pair(const S* p, decltype(ld2(p, 0))& a,
                                        decltype(ld2(p, 0))& b) {
  if constexpr (sizeof(S) == 4) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    S v[2];
    memcpy(v, &u, sizeof(u));
    a = ld2(v, 0);
    b = ld2(v, 1);
  } else if constexpr (sizeof(S) == 8) {
    const float4 u = *reinterpret_cast<const float4*>(p);
    S v[2];
    memcpy(v, &u, sizeof(u));
    a = ld2(v, 0);
    b = ld2(v, 1);
  } else {
    a = ld2(p, 0);
    b = ld2(p, 1);
  }
}
template <class T>
__device__ __forceinline__ void st_pair(C<T>* p, C<T> a, C<T> b) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    p[0] = a;
    p[1] = b;
  }
}

// Fused pre-smoothing, residual and full-weighting restriction for one
// BX x BY tile of coarse nodes and a group of right-hand sides, one thread
// per coarse node (I, J) owning the 2 x 2 fine nodes (2I + a, 2J + b), a, b
// in {0, 1}: their f, x = D^-1 f and residual stay in registers, the
// neighbours come from shared memory as aligned pairs, and the restriction
// exchanges column sums with the thread below (shared memory) and the one to
// the left (warp shuffle).  The fine tile with its halo is [2I0-2, 2I0+2BX]
// x [2J0-2, 2J0+2BY], stored with rows of CW = XW + 1 (even) entries so that
// the pairs of every thread are aligned.  Tiles off the boundary
// (INTERIOR) need no tests; the others zero what lies outside the grid,
// keep Dirichlet boundary nodes at zero and weight the neighbours of
// Sommerfeld boundary rows (nb_code).
template <class T, class SF>
struct PreRestrictCell {
  static constexpr int XW = 2 * BX + 3, XH = 2 * BY + 3, CW = XW + 1;
  static constexpr int NQ = XW * XH, NT = BX * BY, NU = (NQ + NT - 1) / NT;
  static constexpr int NHX = 3 * XW + 3 * 2 * BY;  // halo x entries
  static constexpr int NHR = 2 * BX + 2 * BY + 1;  // halo residual entries
  static constexpr int STAGE = align16(CW * XH * (int)sizeof(SF));
  static constexpr int XS = align16(CW * XH * (int)sizeof(C<T>));
  static constexpr int TR = align16((BY + 1) * 2 * BX * (int)sizeof(C<T>));
  static constexpr int HC = align16((2 * BY + 1) * (int)sizeof(C<T>));
  static constexpr int smem(int ns, int rpb) { return ns * STAGE + XS + TR + HC + 4 * rpb; }
  static_assert(NHX <= NT && NHR <= NT, "halo entries per thread");
};

// residual row of a fine node with neighbour weights code (see nb_code)
template <class T, bool INTERIOR>
__device__ __forceinline__ C<T> resid_row(T ih2, T omc, C<T> f, C<T> xw, C<T> xe, C<T> xs,
                                          C<T> xn, unsigned code) {
  if (INTERIOR) return rfma(ih2, (xw + xe) + (xs + xn), omc * f);
  C<T> a = T(code & 3u) * xw;
  a = rfma(T((code >> 2) & 3u), xe, a);
  a = rfma(T((code >> 4) & 3u), xs, a);
  a = rfma(T((code >> 6) & 3u), xn, a);
  return rfma(ih2, a, omc * f);
}

template <class T, class SF, class SX, class SC, int NS, bool INTERIOR>
__device__ __forceinline__ void pre_restrict_cell_body(
    const LevelDev& Lf, const LevelDev& Lc, int bc, T omc, VRefE<SF> fin, long long frs,
    SX* x, SC* fc, int na, const int* act, unsigned char* smraw) {
  using P = PreRestrictCell<T, SF>;
  constexpr int XW = P::XW, XH = P::XH, CW = P::CW, NQ = P::NQ, NT = P::NT, NU = P::NU;
  constexpr int SV = P::STAGE / (int)sizeof(SF);
  SF* fst = reinterpret_cast<SF*>(smraw);
  C<T>* xs = reinterpret_cast<C<T>*>(smraw + NS * P::STAGE);
  C<T>* tr = reinterpret_cast<C<T>*>(smraw + NS * P::STAGE + P::XS);
  C<T>* hc = reinterpret_cast<C<T>*>(smraw + NS * P::STAGE + P::XS + P::TR);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int I = blockIdx.x * BX + tx, J = blockIdx.y * BY + ty;
  const int fx0 = 2 * blockIdx.x * BX - 2, fy0 = 2 * blockIdx.y * BY - 2;
  const int nfx = Lf.nx, nfy = Lf.ny;
  const long long nf = (long long)nfx * nfy, nc = (long long)Lc.nx * Lc.ny;
  const SF* fbase = fin.get();
  const T ih2 = ih2_of<T>(Lf);
  const C<T>* dinv = dinv_of<T>(Lf);
  // fine node (gi, gj): inside the grid / an unknown (not a Dirichlet
  // boundary node)
  auto in_grid = [&](int gi, int gj) { return gi >= 0 && gi < nfx && gj >= 0 && gj < nfy; };
  auto unknown = [&](int gi, int gj) {
    return INTERIOR || (in_grid(gi, gj) && !(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy)));
  };
  // copies of the tile: global offset of entry q (shared index q + q / XW),
  // -1 outside the grid (zero in every stage)
  int gq[NU];
#pragma unroll
  for (int u = 0; u < NU; ++u) {
    const int q = tid + u * NT;
    const int gi = fx0 + q % XW, gj = fy0 + q / XW;
    gq[u] = q < NQ && (INTERIOR || in_grid(gi, gj)) ? gj * nfx + gi : -1;
    if (!INTERIOR && q < NQ && gq[u] < 0)
      for (int sidx = 0; sidx < NS; ++sidx) fst[sidx * SV + q + q / XW] = szero<SF>();
  }
  // own fine nodes: shared index of (2I, 2J), global index, D^-1 (zero for
  // nodes that are not unknowns, so that their x is zero), and outside the
  // interior: which are inside the grid (x stored), which are unknowns
  // (residual kept) and the neighbour weights of each
  const int o0 = (2 * ty + 2) * CW + 2 * tx + 2;
  const int g00 = (2 * J) * nfx + 2 * I;
  C<T> d[4];
  unsigned ing = 0xfu, unk = 0xfu, code = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int gi = 2 * I + (c & 1), gj = 2 * J + (c >> 1);
    if (!INTERIOR) {
      if (!in_grid(gi, gj)) ing &= ~(1u << c);
      if (!unknown(gi, gj)) unk &= ~(1u << c);
      if (unk >> c & 1u) code |= nb_code(bc, gi, gj, nfx, nfy) << (8 * c);
    }
    d[c] = (unk >> c & 1u) ? dinv[(long long)gj * nfx + gi] : czero<T>();
  }
  // halo x entry of this thread (rows 0, 1, XH-1 of the tile, then columns
  // 0, 1, XW-1 of its inner rows)
  int hxi = -1;
  C<T> hxd = czero<T>();
  if (tid < P::NHX) {
    int lx, ly;
    if (tid < 3 * XW) {
      const int rr = tid / XW;
      lx = tid % XW;
      ly = rr == 2 ? XH - 1 : rr;
    } else {
      const int e = tid - 3 * XW, cc = e / (2 * BY);
      ly = 2 + e % (2 * BY);
      lx = cc == 2 ? XW - 1 : cc;
    }
    hxi = ly * CW + lx;
    if (unknown(fx0 + lx, fy0 + ly)) hxd = dinv[(long long)(fy0 + ly) * nfx + fx0 + lx];
  }
  // halo residual entry: row 2J0-1 (tr row 0) or column 2I0-1 (hc)
  int hri = -1;
  unsigned hcode = 0;
  bool hunk = true;
  if (tid < P::NHR) {
    const int lx = tid < 2 * BX ? tid + 2 : 1, ly = tid < 2 * BX ? 1 : 1 + tid - 2 * BX;
    hri = ly * CW + lx;
    if (!INTERIOR) {
      hunk = unknown(fx0 + lx, fy0 + ly);
      if (hunk) hcode = nb_code(bc, fx0 + lx, fy0 + ly, nfx, nfy);
    }
  }
  // the coarse node: stored (inside the coarse grid), zero (Dirichlet
  // boundary)
  const bool cst = INTERIOR || (I < Lc.nx && J < Lc.ny);
  const bool cdir = !INTERIOR && bc == BC_DIRICHLET && cst && on_bnd(I, J, Lc.nx, Lc.ny);
  auto issue = [&](int k) {
    if (k < na) {
      const SF* fr = fbase + (long long)act[k] * frs;
      SF* stg = fst + (k % NS) * SV;
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        const int q = tid + u * NT;
        if (gq[u] >= 0) cp_async_el<sizeof(SF)>(stg + q + q / XW, fr + gq[u]);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) issue(k);
  for (int k = 0; k < na; ++k) {
    cp_async_wait<NS - 2>();
    __syncthreads();
    issue(k + NS - 1);
    const SF* stg = fst + (k % NS) * SV;
    const int r = act[k];
    // x = D^-1 f: own nodes in registers and shared memory, halo in shared
    C<T> f00, f10, f01, f11;
    ld_pair(stg + o0, f00, f10);
    ld_pair(stg + o0 + CW, f01, f11);
    const C<T> x00 = cmul(d[0], f00), x10 = cmul(d[1], f10);
    const C<T> x01 = cmul(d[2], f01), x11 = cmul(d[3], f11);
    st_pair<T>(xs + o0, x00, x10);
    st_pair<T>(xs + o0 + CW, x01, x11);
    SX* xr = x + (long long)r * nf + g00;
    if (ing & 1u) st2(xr, 0, x00);
    if (ing & 2u) st2(xr, 1, x10);
    if (ing & 4u) st2(xr, nfx, x01);
    if (ing & 8u) st2(xr, nfx + 1, x11);
    if (hxi >= 0) xs[hxi] = cmul(hxd, ld2(stg, hxi));
    __syncthreads();
    // residuals (1 - w) f + (1/h^2) sum of the (weighted) neighbours' x
    C<T> t0, t1, xs0, xs1, xn0, xn1, xw0, xw1, xe0, xe1;
    ld_pair(xs + o0 - CW, xs0, xs1);
    ld_pair(xs + o0 + 2 * CW, xn0, xn1);
    ld_pair(xs + o0 - 2, t0, xw0);
    ld_pair(xs + o0 - 2 + CW, t1, xw1);
    ld_pair(xs + o0 + 2, xe0, t0);
    ld_pair(xs + o0 + 2 + CW, xe1, t1);
    C<T> r00 = resid_row<T, INTERIOR>(ih2, omc, f00, xw0, x10, xs0, x01, code);
    C<T> r10 = resid_row<T, INTERIOR>(ih2, omc, f10, x00, xe0, xs1, x11, code >> 8);
    C<T> r01 = resid_row<T, INTERIOR>(ih2, omc, f01, xw1, x11, x00, xn0, code >> 16);
    C<T> r11 = resid_row<T, INTERIOR>(ih2, omc, f11, x01, xe1, x10, xn1, code >> 24);
    if (!INTERIOR) {
      if (!(unk & 1u)) r00 = czero<T>();
      if (!(unk & 2u)) r10 = czero<T>();
      if (!(unk & 4u)) r01 = czero<T>();
      if (!(unk & 8u)) r11 = czero<T>();
    }
    st_pair<T>(tr + (ty + 1) * 2 * BX + 2 * tx, r01, r11);
    if (hri >= 0) {
      C<T> v = resid_row<T, INTERIOR>(ih2, omc, ld2(stg, hri), xs[hri - 1], xs[hri + 1],
                                      xs[hri - CW], xs[hri + CW], hcode);
      if (!hunk) v = czero<T>();
      if (tid < 2 * BX)
        tr[tid] = v;
      else
        hc[tid - 2 * BX] = v;
    }
    __syncthreads();
    // full weighting: column sums over rows 2J-1..2J+1, then columns
    C<T> s0, s1;
    ld_pair(tr + ty * 2 * BX + 2 * tx, s0, s1);
    s0 = s0 + (T(2) * r00 + r01);
    s1 = s1 + (T(2) * r10 + r11);
    C<T> sw;
    sw.x = __shfl_up_sync(0xffffffffu, s1.x, 1);
    sw.y = __shfl_up_sync(0xffffffffu, s1.y, 1);
    if (tx == 0) sw = (hc[2 * ty] + hc[2 * ty + 2]) + T(2) * hc[2 * ty + 1];
    if (cst)
      st2(fc, r * nc + (long long)J * Lc.nx + I,
          cdir ? czero<T>() : T(0.0625) * ((sw + s1) + T(2) * s0));
  }
  cp_async_wait<0>();
}

template <class T, class SF, class SX, class SC, int NS>
__global__ void __launch_bounds__(BX * BY, 3)
k_pre_restrict_mr(LevelDev Lf, LevelDev Lc, int bc, T omc, VRefE<SF> fin, long long frs,
                  SX* __restrict__ x, SC* __restrict__ fc, int nrhs, int rpb,
                  const int* __restrict__ done, unsigned long long* abytes) {
  using P = PreRestrictCell<T, SF>;
  extern __shared__ __align__(16) unsigned char smraw[];
  int* act = reinterpret_cast<int*>(smraw + P::smem(NS, 0));
  __shared__ int nact_s;
  const int r0 = blockIdx.z * rpb, r1 = min(nrhs, r0 + rpb);
  const int na = list_active(done, r0, r1, act, &nact_s);
  if (na == 0) return;
  if (abytes && threadIdx.x == 0 && threadIdx.y == 0) {
    // algorithmic bytes of the tile: f read and x written per own fine node,
    // the coarse right-hand side written per own coarse node, for each
    // active RHS; D^-1 once per launch
    const long long fw = min(2 * BX, Lf.nx - 2 * (int)blockIdx.x * BX);
    const long long fh = min(2 * BY, Lf.ny - 2 * (int)blockIdx.y * BY);
    const long long cw = min(BX, Lc.nx - (int)blockIdx.x * BX);
    const long long ch = min(BY, Lc.ny - (int)blockIdx.y * BY);
    unsigned long long b = (unsigned long long)na *
        (fw * fh * (sizeof(SF) + sizeof(SX)) + cw * ch * sizeof(SC));
    if (blockIdx.z == 0) b += (unsigned long long)(fw * fh * sizeof(C<T>));
    atomicAdd(abytes, b);
  }
  // the x tile [2I0-2, 2I0+2BX] x [2J0-2, 2J0+2BY] inside the grid and off
  // its boundary rows and columns
  const int fx0 = 2 * blockIdx.x * BX - 2, fy0 = 2 * blockIdx.y * BY - 2;
  const bool interior = fx0 >= 1 && fy0 >= 1 && fx0 + P::XW <= Lf.nx - 1 &&
                        fy0 + P::XH <= Lf.ny - 1;
  if (interior)
    pre_restrict_cell_body<T, SF, SX, SC, NS, true>(Lf, Lc, bc, omc, fin, frs, x, fc, na,
                                                    act, smraw);
  else
    pre_restrict_cell_body<T, SF, SX, SC, NS, false>(Lf, Lc, bc, omc, fin, frs, x, fc, na,
                                                     act, smraw);
}

template <class T, class SC, class SX, class SF, int TXW>
struct ProlongSmoothMR {
  static constexpr int NPX = TXW / BX;
  static constexpr int PW = TXW + 2, PH = BY + 2, NP = PW * PH;
  static constexpr int CW = TXW / 2 + 2, CH = BY / 2 + 2, NC = CW * CH;
  static constexpr int NF = TXW * BY, NT = BX * BY;
  static constexpr int N1 = (NP + NT - 1) / NT, N3 = (NC + NT - 1) / NT;
  static constexpr int OX = 0, OC = align16(NP * (int)sizeof(SX)),
                       OF = OC + align16(NC * (int)sizeof(SC)),
                       STAGE = OF + align16(NF * (int)sizeof(SF));
  static constexpr int XP = align16(NP * (int)sizeof(C<T>));
  static constexpr int smem(int ns, int rpb) { return ns * STAGE + XP + 4 * rpb; }
};

// Fused coarse-grid correction and post-smoothing, xo = x' + D^-1 (f - M x')
// with x' = x + P xc, for one TXW x BY tile of fine nodes and a group of rpb
// right-hand sides (each thread owns TXW / BX nodes of a tile row).
template <class T, class SC, class SX, class SF, class SO, int NS, int TXW, bool INTERIOR>
__device__ __forceinline__ void prolong_smooth_mr_body(
    const LevelDev& Lf, const LevelDev& Lc, int bc, T omc, const SC* xc, const SX* x,
    VRefE<SF> fin, long long frs, SO* xo, int na, const int* act, unsigned char* smraw) {
  using P = ProlongSmoothMR<T, SC, SX, SF, TXW>;
  constexpr int PW = P::PW, NP = P::NP, CW = P::CW, NC = P::NC, NT = P::NT;
  constexpr int N1 = P::N1, N3 = P::N3, NPX = P::NPX;
  C<T>* xp = reinterpret_cast<C<T>*>(smraw + NS * P::STAGE);
  const int i0 = blockIdx.x * TXW, j0 = blockIdx.y * BY;
  const int ic0 = i0 / 2 - 1, jc0 = j0 / 2 - 1;
  const int tid = threadIdx.y * BX + threadIdx.x;
  const int nfx = Lf.nx, nfy = Lf.ny, ncx = Lc.nx, ncy = Lc.ny;
  const long long nf = (long long)nfx * nfy, nc = (long long)ncx * ncy;
  const SF* fbase = fin.get();
  const T ih2 = ih2_of<T>(Lf);
  auto sx_of = [&](int k) {
    return reinterpret_cast<SX*>(smraw + (k % NS) * P::STAGE + P::OX);
  };
  auto sc_of = [&](int k) {
    return reinterpret_cast<SC*>(smraw + (k % NS) * P::STAGE + P::OC);
  };
  auto sf_of = [&](int k) {
    return reinterpret_cast<SF*>(smraw + (k % NS) * P::STAGE + P::OF);
  };
  // x tile with its 1-node halo: node, and the staged coarse values its
  // bilinear interpolation reads (b0, one step right if x is odd, one row
  // down if y is odd; the even directions read the same value twice)
  int gx[N1], cb[N1], cdx[N1], cdy[N1];
  unsigned ing = 0, corr = 0;
#pragma unroll
  for (int u = 0; u < N1; ++u) {
    const int q = tid + u * NT;
    const int gi = i0 - 1 + q % PW, gj = j0 - 1 + q / PW;
    gx[u] = -1;
    cb[u] = 0;
    cdx[u] = 0;
    cdy[u] = 0;
    if (q < NP && gi >= 0 && gi < nfx && gj >= 0 && gj < nfy) {
      gx[u] = gj * nfx + gi;
      ing |= 1u << u;
      if (INTERIOR || !(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy))) corr |= 1u << u;
      cb[u] = ((gj >> 1) - jc0) * CW + ((gi >> 1) - ic0);
      cdx[u] = gi & 1;
      cdy[u] = (gj & 1) * CW;
    }
  }
  int gc[N3];
#pragma unroll
  for (int u = 0; u < N3; ++u) {
    const int q = tid + u * NT;
    const int I = ic0 + q % CW, J = jc0 + q / CW;
    gc[u] = (q < NC && I >= 0 && I < ncx && J >= 0 && J < ncy) ? J * ncx + I : -1;
  }
  // own nodes: D^-1 and neighbour weights in registers, f staged
  int go[NPX];
  unsigned code[NPX];
  unsigned dir = 0;
  C<T> down[NPX];
  const int j = j0 + threadIdx.y;
#pragma unroll
  for (int p = 0; p < NPX; ++p) {
    const int i = i0 + threadIdx.x + p * BX;
    go[p] = (i < nfx && j < nfy) ? j * nfx + i : -1;
    down[p] = go[p] >= 0 ? dinv_of<T>(Lf)[go[p]] : czero<T>();
    code[p] = 0;
    if (go[p] >= 0 && !INTERIOR) {
      if (bc == BC_DIRICHLET && on_bnd(i, j, nfx, nfy))
        dir |= 1u << p;
      else
        code[p] = nb_code(bc, i, j, nfx, nfy);
    }
  }
  for (int sidx = 0; sidx < NS; ++sidx) {
#pragma unroll
    for (int u = 0; u < N1; ++u)
      if (tid + u * NT < NP && gx[u] < 0) sx_of(sidx)[tid + u * NT] = szero<SX>();
#pragma unroll
    for (int u = 0; u < N3; ++u)
      if (tid + u * NT < NC && gc[u] < 0) sc_of(sidx)[tid + u * NT] = szero<SC>();
#pragma unroll
    for (int p = 0; p < NPX; ++p)
      if (go[p] < 0) sf_of(sidx)[threadIdx.y * TXW + threadIdx.x + p * BX] = szero<SF>();
  }
  auto issue = [&](int k) {
    if (k < na) {
      const int r = act[k];
      const SX* xr = x + (long long)r * nf;
      const SC* xcr = xc + (long long)r * nc;
      const SF* fr = fbase + (long long)r * frs;
      SX* sx = sx_of(k);
      SC* sc = sc_of(k);
      SF* sf = sf_of(k);
#pragma unroll
      for (int u = 0; u < N1; ++u)
        if (gx[u] >= 0) cp_async_el<sizeof(SX)>(sx + tid + u * NT, xr + gx[u]);
#pragma unroll
      for (int u = 0; u < N3; ++u)
        if (gc[u] >= 0) cp_async_el<sizeof(SC)>(sc + tid + u * NT, xcr + gc[u]);
#pragma unroll
      for (int p = 0; p < NPX; ++p)
        if (go[p] >= 0)
          cp_async_el<sizeof(SF)>(sf + threadIdx.y * TXW + threadIdx.x + p * BX, fr + go[p]);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) issue(k);
  for (int k = 0; k < na; ++k) {
    cp_async_wait<NS - 2>();
    __syncthreads();
    issue(k + NS - 1);
    const SX* sx = sx_of(k);
    const SC* sc = sc_of(k);
    const SF* sf = sf_of(k);
    const int r = act[k];
#pragma unroll
    for (int u = 0; u < N1; ++u) {
      const int q = tid + u * NT;
      if (q < NP) {
        C<T> v = czero<T>();
        if (ing >> u & 1u) {
          v = ld2(sx, q);
          if (corr >> u & 1u) {
            const int b0 = cb[u], b1 = cb[u] + cdy[u];
            const C<T> a = T(0.5) * (ld2(sc, b0) + ld2(sc, b0 + cdx[u]));
            const C<T> c = T(0.5) * (ld2(sc, b1) + ld2(sc, b1 + cdx[u]));
            v = v + T(0.5) * (a + c);
          }
        }
        xp[q] = v;
      }
    }
    __syncthreads();
    SO* orow = xo + (long long)r * nf;
#pragma unroll
    for (int p = 0; p < NPX; ++p) {
      if (go[p] < 0) continue;
      if (!INTERIOR && (dir >> p & 1u)) {
        st2(orow, go[p], czero<T>());
        continue;
      }
      const int c = (threadIdx.y + 1) * PW + (threadIdx.x + p * BX + 1);
      const C<T> g =
          rfma(ih2, nb_sum<T, INTERIOR>(xp, c, PW, code[p]),
               ld2(sf, threadIdx.y * TXW + threadIdx.x + p * BX));
      st2(orow, go[p], cfma(down[p], g, omc * xp[c]));
    }
  }
  cp_async_wait<0>();
}

template <class T, class SC, class SX, class SF, class SO, int NS, int TXW>
__global__ void __launch_bounds__(BX * BY)
k_prolong_smooth_mr(LevelDev Lf, LevelDev Lc, int bc, T omc, const SC* __restrict__ xc,
                    const SX* __restrict__ x, VRefE<SF> fin, long long frs,
                    SO* __restrict__ xo, int nrhs, int rpb, const int* __restrict__ done,
                    unsigned long long* abytes) {
  using P = ProlongSmoothMR<T, SC, SX, SF, TXW>;
  extern __shared__ __align__(16) unsigned char smraw[];
  int* act = reinterpret_cast<int*>(smraw + NS * P::STAGE + P::XP);
  __shared__ int nact_s;
  const int r0 = blockIdx.z * rpb, r1 = min(nrhs, r0 + rpb);
  const int na = list_active(done, r0, r1, act, &nact_s);
  if (na == 0) return;
  if (abytes && threadIdx.x == 0 && threadIdx.y == 0) {
    // algorithmic bytes of the tile: x and f read and the result written per
    // own fine node, the correction read per coarse node under the tile
    // (the tile's fine nodes with both indices even), for each active RHS;
    // D^-1 once per launch
    const long long fw = min(TXW, Lf.nx - (int)blockIdx.x * TXW);
    const long long fh = min(BY, Lf.ny - (int)blockIdx.y * BY);
    unsigned long long b = (unsigned long long)na *
        (fw * fh * (sizeof(SX) + sizeof(SF) + sizeof(SO)) +
         ((fw + 1) / 2) * ((fh + 1) / 2) * sizeof(SC));
    if (blockIdx.z == 0) b += (unsigned long long)(fw * fh * sizeof(C<T>));
    atomicAdd(abytes, b);
  }
  // the x' tile [i0-1, i0+TXW] x [j0-1, j0+BY] inside the grid and off its
  // boundary rows and columns
  const int fx0 = blockIdx.x * TXW - 1, fy0 = blockIdx.y * BY - 1;
  const bool interior = fx0 >= 1 && fy0 >= 1 && fx0 + P::PW <= Lf.nx - 1 &&
                        fy0 + P::PH <= Lf.ny - 1;
  if (interior)
    prolong_smooth_mr_body<T, SC, SX, SF, SO, NS, TXW, true>(Lf, Lc, bc, omc, xc, x, fin,
                                                             frs, xo, na, act, smraw);
  else
    prolong_smooth_mr_body<T, SC, SX, SF, SO, NS, TXW, false>(Lf, Lc, bc, omc, xc, x, fin,
                                                              frs, xo, na, act, smraw);
}

// Fused coarse-grid correction and post-smoothing with one thread per
// coarse cell (I, J) owning the fine nodes (2I + a, 2J + b), a, b in {0, 1}:
// x' = x + P xc for them from the four coarse values of the cell, kept in
// registers, then xo = (1 - w) x' + D^-1 (f + (1/h^2) sum of the weighted
// neighbours' x'), the neighbours from shared memory as aligned pairs.  A
// block covers 2BX x 2BY fine nodes; x' is staged with a one-node halo in
// rows of CW = 2BX + 4 entries whose column 0 (node i0 - 2) is unused, so
// that the pairs of every thread are aligned.  INTERIOR as for the
// restriction.
template <class T, class SC, class SX, class SF>
struct ProlongSmoothCell {
  static constexpr int FW = 2 * BX, FH = 2 * BY;        // own fine nodes
  static constexpr int CW = FW + 4, XH = FH + 2;        // x / x' tile rows
  static constexpr int QW = FW + 2, NQ = QW * XH;       // x entries copied
  static constexpr int KW = BX + 2, KH = BY + 2, NK = KW * KH;  // coarse entries
  static constexpr int NT = BX * BY, NU = (NQ + NT - 1) / NT, NV = (NK + NT - 1) / NT;
  static constexpr int NHX = 2 * QW + 2 * FH;           // halo x' entries
  static constexpr int OC = align16(CW * XH * (int)sizeof(SX));
  static constexpr int OF = OC + align16(NK * (int)sizeof(SC));
  static constexpr int STAGE = OF + align16(FW * FH * (int)sizeof(SF));
  static constexpr int XP = align16(CW * XH * (int)sizeof(C<T>));
  static constexpr int smem(int ns, int rpb) { return ns * STAGE + XP + 4 * rpb; }
  static_assert(NHX <= NT, "halo entries per thread");
};

template <class T, class SC, class SX, class SF, class SO, int NS, bool INTERIOR>
__device__ __forceinline__ void prolong_smooth_cell_body(
    const LevelDev& Lf, const LevelDev& Lc, int bc, T omc, const SC* xc, const SX* x,
    VRefE<SF> fin, long long frs, SO* xo, int na, const int* act, unsigned char* smraw) {
  using P = ProlongSmoothCell<T, SC, SX, SF>;
  constexpr int FW = P::FW, CW = P::CW, QW = P::QW, NQ = P::NQ, KW = P::KW, NK = P::NK;
  constexpr int NT = P::NT, NU = P::NU, NV = P::NV;
  C<T>* xp = reinterpret_cast<C<T>*>(smraw + NS * P::STAGE);
  auto sx_of = [&](int k) { return reinterpret_cast<SX*>(smraw + (k % NS) * P::STAGE); };
  auto sc_of = [&](int k) {
    return reinterpret_cast<SC*>(smraw + (k % NS) * P::STAGE + P::OC);
  };
  auto sf_of = [&](int k) {
    return reinterpret_cast<SF*>(smraw + (k % NS) * P::STAGE + P::OF);
  };
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int I0 = blockIdx.x * BX, J0 = blockIdx.y * BY;
  const int i0 = 2 * I0, j0 = 2 * J0;     // first own fine node
  const int I = I0 + tx, J = J0 + ty;
  const int nfx = Lf.nx, nfy = Lf.ny, ncx = Lc.nx, ncy = Lc.ny;
  const long long nf = (long long)nfx * nfy, nc = (long long)ncx * ncy;
  const SF* fbase = fin.get();
  const T ih2 = ih2_of<T>(Lf);
  const C<T>* dinv = dinv_of<T>(Lf);
  auto in_grid = [&](int gi, int gj) { return gi >= 0 && gi < nfx && gj >= 0 && gj < nfy; };
  auto dir_bnd = [&](int gi, int gj) {
    return !INTERIOR && bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy);
  };
  // copies: x over [i0-1, i0+FW] x [j0-1, j0+FH] (tile column 1 on), the
  // coarse correction over [I0-1, I0+BX] x [J0-1, J0+BY], f over the own
  // nodes; -1 outside the grid (zero in every stage)
  int gx[NU], gc[NV];
#pragma unroll
  for (int u = 0; u < NU; ++u) {
    const int q = tid + u * NT;
    const int gi = i0 - 1 + q % QW, gj = j0 - 1 + q / QW;
    gx[u] = q < NQ && (INTERIOR || in_grid(gi, gj)) ? gj * nfx + gi : -1;
  }
#pragma unroll
  for (int u = 0; u < NV; ++u) {
    const int q = tid + u * NT;
    const int ci = I0 - 1 + q % KW, cj = J0 - 1 + q / KW;
    gc[u] = q < NK && (INTERIOR || (ci >= 0 && ci < ncx && cj >= 0 && cj < ncy))
                ? cj * ncx + ci
                : -1;
  }
  // own nodes: shared index of (2I, 2J) in the x tile, global index, D^-1,
  // and outside the interior: inside the grid (stored), Dirichlet boundary
  // (stored as zero, no correction), neighbour weights
  const int o0 = (2 * ty + 1) * CW + 2 * tx + 2;
  const int of0 = (2 * ty) * FW + 2 * tx;
  const int k0 = (ty + 1) * KW + tx + 1;
  const int g00 = (2 * J) * nfx + 2 * I;
  C<T> d[4];
  unsigned ing = 0xfu, dir = 0, code = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int gi = 2 * I + (c & 1), gj = 2 * J + (c >> 1);
    if (!INTERIOR) {
      if (!in_grid(gi, gj)) ing &= ~(1u << c);
      else if (dir_bnd(gi, gj)) dir |= 1u << c;
      else code |= nb_code(bc, gi, gj, nfx, nfy) << (8 * c);
    }
    d[c] = (ing >> c & 1u) ? dinv[(long long)gj * nfx + gi] : czero<T>();
  }
  // halo x' entry of this thread (tile rows 0 and XH-1 over columns 1..QW,
  // then columns 1 and QW of the inner rows): shared index, coarse base
  // index and steps of the bilinear interpolation, inside the grid,
  // corrected
  int hxi = -1, hcb = 0, hdx = 0, hdy = 0;
  bool hin = true, hcor = true;
  if (tid < P::NHX) {
    int lx, ly;
    if (tid < 2 * QW) {
      lx = 1 + tid % QW;
      ly = tid < QW ? 0 : P::XH - 1;
    } else {
      const int e = tid - 2 * QW;
      ly = 1 + e % P::FH;
      lx = e < P::FH ? 1 : QW;
    }
    const int gi = i0 - 2 + lx, gj = j0 - 1 + ly;
    hxi = ly * CW + lx;
    if (!INTERIOR) {
      hin = in_grid(gi, gj);
      hcor = hin && !dir_bnd(gi, gj);
    }
    hcb = ((gj >> 1) - (J0 - 1)) * KW + ((gi >> 1) - (I0 - 1));
    hdx = gi & 1;
    hdy = (gj & 1) * KW;
  }
  if (!INTERIOR) {
    for (int sidx = 0; sidx < NS; ++sidx) {
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        const int q = tid + u * NT;
        if (q < NQ && gx[u] < 0) sx_of(sidx)[(q / QW) * CW + 1 + q % QW] = szero<SX>();
      }
#pragma unroll
      for (int u = 0; u < NV; ++u) {
        const int q = tid + u * NT;
        if (q < NK && gc[u] < 0) sc_of(sidx)[q] = szero<SC>();
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (!(ing >> c & 1u)) sf_of(sidx)[of0 + (c >> 1) * FW + (c & 1)] = szero<SF>();
    }
  }
  auto issue = [&](int k) {
    if (k < na) {
      const int r = act[k];
      const SX* xr = x + (long long)r * nf;
      const SC* xcr = xc + (long long)r * nc;
      const SF* fr = fbase + (long long)r * frs + g00;
      SX* sx = sx_of(k);
      SC* sc = sc_of(k);
      SF* sf = sf_of(k);
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        const int q = tid + u * NT;
        if (gx[u] >= 0) cp_async_el<sizeof(SX)>(sx + (q / QW) * CW + 1 + q % QW, xr + gx[u]);
      }
#pragma unroll
      for (int u = 0; u < NV; ++u)
        if (gc[u] >= 0) cp_async_el<sizeof(SC)>(sc + tid + u * NT, xcr + gc[u]);
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (ing >> c & 1u)
          cp_async_el<sizeof(SF)>(sf + of0 + (c >> 1) * FW + (c & 1),
                                  fr + (c >> 1) * nfx + (c & 1));
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) issue(k);
  for (int k = 0; k < na; ++k) {
    cp_async_wait<NS - 2>();
    __syncthreads();
    issue(k + NS - 1);
    const SX* sx = sx_of(k);
    const SC* sc = sc_of(k);
    const SF* sf = sf_of(k);
    const int r = act[k];
    // x' = x + P xc: own nodes (registers and shared memory), halo
    C<T> x00, x10, x01, x11;
    ld_pair(sx + o0, x00, x10);
    ld_pair(sx + o0 + CW, x01, x11);
    {
      const C<T> c00 = ld2(sc, k0), c10 = ld2(sc, k0 + 1);
      const C<T> c01 = ld2(sc, k0 + KW), c11 = ld2(sc, k0 + KW + 1);
      const C<T> h0 = T(0.5) * (c00 + c10), h1 = T(0.5) * (c01 + c11);
      const C<T> v0 = T(0.5) * (c00 + c01);
      if (INTERIOR || !(dir & 1u)) x00 = x00 + c00;
      if (INTERIOR || !(dir & 2u)) x10 = x10 + h0;
      if (INTERIOR || !(dir & 4u)) x01 = x01 + v0;
      if (INTERIOR || !(dir & 8u)) x11 = x11 + T(0.5) * (h0 + h1);
      if (!INTERIOR) {
        if (!(ing & 1u)) x00 = czero<T>();
        if (!(ing & 2u)) x10 = czero<T>();
        if (!(ing & 4u)) x01 = czero<T>();
        if (!(ing & 8u)) x11 = czero<T>();
      }
    }
    st_pair<T>(xp + o0, x00, x10);
    st_pair<T>(xp + o0 + CW, x01, x11);
    if (hxi >= 0) {
      C<T> v = ld2(sx, hxi);
      if (hcor) {
        const int b1 = hcb + hdy;
        const C<T> a = T(0.5) * (ld2(sc, hcb) + ld2(sc, hcb + hdx));
        const C<T> c = T(0.5) * (ld2(sc, b1) + ld2(sc, b1 + hdx));
        v = v + T(0.5) * (a + c);
      }
      xp[hxi] = hin ? v : czero<T>();
    }
    __syncthreads();
    // xo = (1 - w) x' + D^-1 (f + (1/h^2) sum of the neighbours' x')
    C<T> t0, t1, xs0, xs1, xn0, xn1, xw0, xw1, xe0, xe1, f00, f10, f01, f11;
    ld_pair(xp + o0 - CW, xs0, xs1);
    ld_pair(xp + o0 + 2 * CW, xn0, xn1);
    ld_pair(xp + o0 - 2, t0, xw0);
    ld_pair(xp + o0 - 2 + CW, t1, xw1);
    ld_pair(xp + o0 + 2, xe0, t0);
    ld_pair(xp + o0 + 2 + CW, xe1, t1);
    ld_pair(sf + of0, f00, f10);
    ld_pair(sf + of0 + FW, f01, f11);
    const C<T> y00 = cfma(d[0], resid_row<T, INTERIOR>(ih2, T(1), f00, xw0, x10, xs0, x01, code),
                          omc * x00);
    const C<T> y10 =
        cfma(d[1], resid_row<T, INTERIOR>(ih2, T(1), f10, x00, xe0, xs1, x11, code >> 8),
             omc * x10);
    const C<T> y01 =
        cfma(d[2], resid_row<T, INTERIOR>(ih2, T(1), f01, xw1, x11, x00, xn0, code >> 16),
             omc * x01);
    const C<T> y11 =
        cfma(d[3], resid_row<T, INTERIOR>(ih2, T(1), f11, x01, xe1, x10, xn1, code >> 24),
             omc * x11);
    SO* orow = xo + (long long)r * nf + g00;
    if (INTERIOR) {
      st2(orow, 0, y00);
      st2(orow, 1, y10);
      st2(orow, nfx, y01);
      st2(orow, nfx + 1, y11);
    } else {
      if (ing & 1u) st2(orow, 0, (dir & 1u) ? czero<T>() : y00);
      if (ing & 2u) st2(orow, 1, (dir & 2u) ? czero<T>() : y10);
      if (ing & 4u) st2(orow, nfx, (dir & 4u) ? czero<T>() : y01);
      if (ing & 8u) st2(orow, nfx + 1, (dir & 8u) ? czero<T>() : y11);
    }
  }
  cp_async_wait<0>();
}

template <class T, class SC, class SX, class SF, class SO, int NS>
__global__ void __launch_bounds__(BX * BY, 3)
k_prolong_smooth_cell(LevelDev Lf, LevelDev Lc, int bc, T omc, const SC* __restrict__ xc,
                      const SX* __restrict__ x, VRefE<SF> fin, long long frs,
                      SO* __restrict__ xo, int nrhs, int rpb, const int* __restrict__ done,
                      unsigned long long* abytes) {
  using P = ProlongSmoothCell<T, SC, SX, SF>;
  extern __shared__ __align__(16) unsigned char smraw[];
  int* act = reinterpret_cast<int*>(smraw + P::smem(NS, 0));
  __shared__ int nact_s;
  const int r0 = blockIdx.z * rpb, r1 = min(nrhs, r0 + rpb);
  const int na = list_active(done, r0, r1, act, &nact_s);
  if (na == 0) return;
  if (abytes && threadIdx.x == 0 && threadIdx.y == 0) {
    // algorithmic bytes as for k_prolong_smooth_mr, over this block's tile
    const long long fw = min(P::FW, Lf.nx - (int)blockIdx.x * P::FW);
    const long long fh = min(P::FH, Lf.ny - (int)blockIdx.y * P::FH);
    unsigned long long b = (unsigned long long)na *
        (fw * fh * (sizeof(SX) + sizeof(SF) + sizeof(SO)) +
         ((fw + 1) / 2) * ((fh + 1) / 2) * sizeof(SC));
    if (blockIdx.z == 0) b += (unsigned long long)(fw * fh * sizeof(C<T>));
    atomicAdd(abytes, b);
  }
  // the x' tile [i0-1, i0+FW] x [j0-1, j0+FH] inside the grid and off its
  // boundary rows and columns
  const int fx0 = blockIdx.x * P::FW - 1, fy0 = blockIdx.y * P::FH - 1;
  const bool interior = fx0 >= 1 && fy0 >= 1 && fx0 + P::FW + 2 <= Lf.nx - 1 &&
                        fy0 + P::FH + 2 <= Lf.ny - 1;
  if (interior)
    prolong_smooth_cell_body<T, SC, SX, SF, SO, NS, true>(Lf, Lc, bc, omc, xc, x, fin, frs,
                                                          xo, na, act, smraw);
  else
    prolong_smooth_cell_body<T, SC, SX, SF, SO, NS, false>(Lf, Lc, bc, omc, xc, x, fin, frs,
                                                           xo, na, act, smraw);
}

// The levels from one with few nodes down to the coarsest, for one right-hand
// side per block, every level's f, x and a scratch vector in shared memory:
// the same steps as the staged kernels (x = D^-1 f, residual (1 - w) f +
// (1/h^2) sum of the weighted neighbours, full weighting; the dense solve;
// x' = x + P xc, then (1 - w) x' + D^-1 (f + (1/h^2) sum of the neighbours'
// x')), one block barrier between steps instead of a launch per step, and
// the intermediate levels kept in FP32.  f is read from and x written to
// the first of these levels' vectors (stored as SL).
template <class SL>
__global__ void __launch_bounds__(512)
k_vcycle_small(const __grid_constant__ SmallLevels d, const SL* __restrict__ fin,
               SL* __restrict__ xout, const float2* __restrict__ minv,
               const int* __restrict__ done) {
  extern __shared__ __align__(16) float2 sm[];
  const int r = blockIdx.x;
  if (done && done[r]) return;
  const int tid = threadIdx.x, nth = blockDim.x, bc = d.bc;
  const float omc = d.omc;
  auto dir_bnd = [&](int i, int j, int nx, int ny) {
    return bc == BC_DIRICHLET && on_bnd(i, j, nx, ny);
  };
  {
    const long long n0 = (long long)d.lv[0].nx * d.lv[0].ny;
    float2* F = sm + d.off[0];
    for (int i = tid; i < n0; i += nth) F[i] = ld2(fin + r * n0, i);
  }
  __syncthreads();
  for (int k = 0; k + 1 < d.nlev; ++k) {
    const LevelDev& L = d.lv[k];
    const int nx = L.nx, ny = L.ny, n = nx * ny;
    float2* F = sm + d.off[k];
    float2* X = F + n;
    float2* T = X + n;
    const float2* dinv = dinv_of<float>(L);
    const float ih2 = ih2_of<float>(L);
    for (int i = tid; i < n; i += nth) {
      const int gi = i % nx, gj = i / nx;
      X[i] = dir_bnd(gi, gj, nx, ny) ? czero<float>() : cmul(dinv[i], F[i]);
    }
    __syncthreads();
    for (int i = tid; i < n; i += nth) {
      const int gi = i % nx, gj = i / nx;
      float2 v = czero<float>();
      if (!dir_bnd(gi, gj, nx, ny)) {
        const float2 xw = gi > 0 ? X[i - 1] : czero<float>();
        const float2 xe = gi < nx - 1 ? X[i + 1] : czero<float>();
        const float2 xs = gj > 0 ? X[i - nx] : czero<float>();
        const float2 xn = gj < ny - 1 ? X[i + nx] : czero<float>();
        v = resid_row<float, false>(ih2, omc, F[i], xw, xe, xs, xn,
                                    nb_code(bc, gi, gj, nx, ny));
      }
      T[i] = v;
    }
    __syncthreads();
    const LevelDev& Lc = d.lv[k + 1];
    const int ncx = Lc.nx, ncy = Lc.ny, nc = ncx * ncy;
    float2* Fc = sm + d.off[k + 1];
    for (int I = tid; I < nc; I += nth) {
      const int ci = I % ncx, cj = I / ncx;
      float2 acc = czero<float>();
      if (!dir_bnd(ci, cj, ncx, ncy)) {
        for (int b = -1; b <= 1; ++b) {
          const int jf = 2 * cj + b;
          if (jf < 0 || jf >= ny) continue;
          const float wb = b == 0 ? 2.f : 1.f;
          for (int a = -1; a <= 1; ++a) {
            const int ifn = 2 * ci + a;
            if (ifn < 0 || ifn >= nx) continue;
            acc = rfma((a == 0 ? 2.f : 1.f) * wb, T[jf * nx + ifn], acc);
          }
        }
        acc = 0.0625f * acc;
      }
      Fc[I] = acc;
    }
    __syncthreads();
  }
  {
    const int n = d.nL;
    const float2* F = sm + d.off[d.nlev - 1];
    float2* X = sm + d.off[d.nlev - 1] + n;
    for (int i = tid; i < n; i += nth) {
      float2 acc = czero<float>();
      const float2* mr = minv + (long long)i * n;
      for (int c = 0; c < n; ++c) acc = cfma(mr[c], F[c], acc);
      X[i] = acc;
    }
  }
  __syncthreads();
  for (int k = d.nlev - 2; k >= 0; --k) {
    const LevelDev& L = d.lv[k];
    const LevelDev& Lc = d.lv[k + 1];
    const int nx = L.nx, ny = L.ny, n = nx * ny;
    float2* F = sm + d.off[k];
    float2* X = F + n;
    float2* T = X + n;
    const float2* Xc = sm + d.off[k + 1] + Lc.nx * Lc.ny;
    const float2* dinv = dinv_of<float>(L);
    const float ih2 = ih2_of<float>(L);
    for (int i = tid; i < n; i += nth) {
      const int gi = i % nx, gj = i / nx;
      float2 v = X[i];
      if (!dir_bnd(gi, gj, nx, ny)) v = v + interp_bilinear<float>(Lc, Xc, gi, gj);
      T[i] = v;
    }
    __syncthreads();
    for (int i = tid; i < n; i += nth) {
      const int gi = i % nx, gj = i / nx;
      float2 v = czero<float>();
      if (!dir_bnd(gi, gj, nx, ny)) {
        const float2 xw = gi > 0 ? T[i - 1] : czero<float>();
        const float2 xe = gi < nx - 1 ? T[i + 1] : czero<float>();
        const float2 xs = gj > 0 ? T[i - nx] : czero<float>();
        const float2 xn = gj < ny - 1 ? T[i + nx] : czero<float>();
        v = cfma(dinv[i],
                 resid_row<float, false>(ih2, 1.f, F[i], xw, xe, xs, xn,
                                         nb_code(bc, gi, gj, nx, ny)),
                 omc * T[i]);
      }
      X[i] = v;
    }
    __syncthreads();
  }
  {
    const long long n0 = (long long)d.lv[0].nx * d.lv[0].ny;
    const float2* X = sm + d.off[0] + n0;
    for (int i = tid; i < n0; i += nth) st2(xout + r * n0, i, X[i]);
  }
}

// x = Minv f on the coarsest level (dense inverse built at setup)
template <class T, class SF, class SO>
__global__ void k_dense_mv(int n, const C<T>* __restrict__ minv, VRefE<SF> fin,
                           SO* __restrict__ x, const int* __restrict__ done) {
  extern __shared__ unsigned char smraw[];
  C<T>* fs = reinterpret_cast<C<T>*>(smraw);
  const int r = blockIdx.y;
  if (done && done[r]) return;
  const SF* f = fin.get();
  for (int c = threadIdx.x; c < n; c += blockDim.x) fs[c] = ld2(f, (long long)r * n + c);
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const C<T>* mr = minv + (long long)row * n;
  C<T> acc = czero<T>();
  for (int c = 0; c < n; ++c) acc = cfma(mr[c], fs[c], acc);
  st2(x, (long long)r * n + row, acc);
}

}  // namespace

template <class T, class SF, class SX>
void launch_jacobi0(const LevelDev& L, int bc, VRefE<SF> f, SX* x, int nrhs,
                    const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_jacobi0<T, SF, SX><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(L, bc, f, x,
                                                                       done);
}
template <class T, class SF, class SX, class SC>
void launch_resid_restrict(const LevelDev& Lf, const LevelDev& Lc, int bc, Shift s,
                           VRefE<SF> f, const SX* x, SC* fc, int nrhs,
                           const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_resid_restrict<T, SF, SX, SC><<<grid2d(Lc.nx, Lc.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, (T)s.re, (T)s.im, f, x, fc, done);
}
template <class T, class SC, class SX>
void launch_prolong_add(const LevelDev& Lf, const LevelDev& Lc, int bc, const SC* xc,
                        SX* x, int nrhs, const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_prolong_add<T, SC, SX><<<grid2d(Lf.nx, Lf.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, xc, x, done);
}
template <class T, class SF, class SX, class SO>
void launch_smooth(const LevelDev& L, int bc, Shift s, VRefE<SF> f, const SX* x,
                   SO* xo, int nrhs, const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_smooth<T, SF, SX, SO><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(
      L, bc, (T)s.re, (T)s.im, f, x, xo, done);
}
template <class T, class SF, class SX, class SC>
void launch_pre_restrict(const LevelDev& Lf, const LevelDev& Lc, int bc, Shift s,
                         VRefE<SF> f, SX* x, SC* fc, int nrhs, const int* done,
                         cudaStream_t st) {
  HZ_COUNT();
  k_pre_restrict<T, SF, SX, SC><<<grid2d(Lc.nx, Lc.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, (T)s.re, (T)s.im, f, x, fc, done);
}
template <class T, class SC, class SX, class SF, class SO>
void launch_prolong_smooth(const LevelDev& Lf, const LevelDev& Lc, int bc, Shift s,
                           const SC* xc, const SX* x, VRefE<SF> f, SO* xo, int nrhs,
                           const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_prolong_smooth<T, SC, SX, SF, SO><<<grid2d(Lf.nx, Lf.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, (T)s.re, (T)s.im, xc, x, f, xo, done);
}
// Multi-RHS staged kernels: grid (tiles, ceil(nrhs / rpb)); the dynamic
// shared memory (the stage ring, the tile, the active-RHS list) is allowed
// up to its largest size once per instantiation.
constexpr int kPreNS = 3, kProNS = 4;

inline int clamp_rpb(int rpb, int nrhs) { return (rpb <= 0 || rpb > nrhs) ? nrhs : rpb; }

// SMs of the current device (looked up once per device)
inline int sm_count_current() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = n > 0 ? n : 1;
  }
  return cache[dev];
}
// Right-hand sides per block of a staged launch: the tuned rpb (clamped),
// halved while the level has too few tiles for two blocks per SM, so that
// the small levels run their right-hand sides side by side instead of one
// after another in a few blocks.
inline int level_rpb(int rpb, long long tiles, int nrhs) {
  rpb = clamp_rpb(rpb, nrhs);
  const long long want = 2LL * sm_count_current();
  while (rpb > 1 && tiles * ((nrhs + rpb - 1) / rpb) < want) rpb = (rpb + 1) / 2;
  return rpb;
}

template <class T, class SF, class SX, class SC>
void launch_pre_restrict_mr(const LevelDev& Lf, const LevelDev& Lc, int bc, double omega,
                            VRefE<SF> f, SX* x, SC* fc, int nrhs, int rpb, const int* done,
                            cudaStream_t st, unsigned long long* abytes, long long frs) {
  HZ_COUNT();
  auto kern = k_pre_restrict_mr<T, SF, SX, SC, kPreNS>;
  static std::once_flag once;
  std::call_once(once, [&] {
    cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         PreRestrictCell<T, SF>::smem(kPreNS, 1024));
  });
  rpb = level_rpb(rpb, (long long)((Lc.nx + BX - 1) / BX) * ((Lc.ny + BY - 1) / BY), nrhs);
  const dim3 grid((Lc.nx + BX - 1) / BX, (Lc.ny + BY - 1) / BY, (nrhs + rpb - 1) / rpb);
  if (frs <= 0) frs = (long long)Lf.nx * Lf.ny;
  kern<<<grid, dim3(BX, BY), PreRestrictCell<T, SF>::smem(kPreNS, rpb), st>>>(
      Lf, Lc, bc, (T)(1.0 - omega), f, frs, x, fc, nrhs, rpb, done, abytes);
}

template <class T, class SC, class SX, class SF, class SO, int TXW>
void launch_prolong_smooth_mr_w(const LevelDev& Lf, const LevelDev& Lc, int bc, double omega,
                                const SC* xc, const SX* x, VRefE<SF> f, SO* xo, int nrhs,
                                int rpb, const int* done, cudaStream_t st,
                                unsigned long long* abytes, long long frs) {
  using P = ProlongSmoothMR<T, SC, SX, SF, TXW>;
  auto kern = k_prolong_smooth_mr<T, SC, SX, SF, SO, kProNS, TXW>;
  static std::once_flag once;
  std::call_once(once, [&] {
    cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         P::smem(kProNS, 1024));
  });
  rpb = level_rpb(rpb, (long long)((Lf.nx + TXW - 1) / TXW) * ((Lf.ny + BY - 1) / BY), nrhs);
  const dim3 grid((Lf.nx + TXW - 1) / TXW, (Lf.ny + BY - 1) / BY, (nrhs + rpb - 1) / rpb);
  if (frs <= 0) frs = (long long)Lf.nx * Lf.ny;
  kern<<<grid, dim3(BX, BY), P::smem(kProNS, rpb), st>>>(Lf, Lc, bc, (T)(1.0 - omega), xc,
                                                         x, f, frs, xo, nrhs, rpb, done,
                                                         abytes);
}

// tile 0: 32 x 8 fine nodes per block, 1: 64 x 8
template <class T, class SC, class SX, class SF, class SO>
void launch_prolong_smooth_mr(const LevelDev& Lf, const LevelDev& Lc, int bc, double omega,
                              const SC* xc, const SX* x, VRefE<SF> f, SO* xo, int nrhs,
                              int rpb, int tile, const int* done, cudaStream_t st,
                              unsigned long long* abytes, long long frs) {
  HZ_COUNT();
  if (tile == 1) {
    using P = ProlongSmoothCell<T, SC, SX, SF>;
    auto kern = k_prolong_smooth_cell<T, SC, SX, SF, SO, kProNS>;
    static std::once_flag once;
    std::call_once(once, [&] {
      cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           P::smem(kProNS, 1024));
    });
    rpb = level_rpb(rpb, (long long)((Lf.nx + P::FW - 1) / P::FW) * ((Lf.ny + P::FH - 1) / P::FH),
                    nrhs);
    const dim3 grid((Lf.nx + P::FW - 1) / P::FW, (Lf.ny + P::FH - 1) / P::FH,
                    (nrhs + rpb - 1) / rpb);
    if (frs <= 0) frs = (long long)Lf.nx * Lf.ny;
    kern<<<grid, dim3(BX, BY), P::smem(kProNS, rpb), st>>>(Lf, Lc, bc, (T)(1.0 - omega), xc,
                                                           x, f, frs, xo, nrhs, rpb, done,
                                                           abytes);
  } else
    launch_prolong_smooth_mr_w<T, SC, SX, SF, SO, BX>(Lf, Lc, bc, omega, xc, x, f, xo, nrhs,
                                                      rpb, done, st, abytes, frs);
}

template <class SL>
void launch_vcycle_small(const SmallLevels& d, const SL* f, SL* x, const float2* minv,
                         int nrhs, const int* done, cudaStream_t st) {
  HZ_COUNT();
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute((const void*)k_vcycle_small<SL>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallLevelBytes);
  });
  k_vcycle_small<SL><<<nrhs, 512, d.bytes, st>>>(d, f, x, minv, done);
}
template void launch_vcycle_small<float2>(const SmallLevels&, const float2*, float2*,
                                          const float2*, int, const int*, cudaStream_t);
template void launch_vcycle_small<__nv_bfloat162>(const SmallLevels&, const __nv_bfloat162*,
                                                  __nv_bfloat162*, const float2*, int,
                                                  const int*, cudaStream_t);

template <class T, class SF, class SO>
void launch_dense_mv(int n, const C<T>* minv, VRefE<SF> f, SO* x, int nrhs,
                     const int* done, cudaStream_t st) {
  HZ_COUNT();
  const int nt = 128;
  k_dense_mv<T, SF, SO><<<dim3((n + nt - 1) / nt, nrhs), nt, n * sizeof(C<T>), st>>>(
      n, minv, f, x, done);
}

// Instantiations: the plain FP64 and FP32 hierarchies (one storage type), and
// the BF16-storage hierarchy under an FP32 V-cycle whose entry vector and
// result stay FP32.
#define HZ_VC_SAME(T)                                                           \
  template void launch_jacobi0<T, C<T>, C<T>>(const LevelDev&, int, VRef<T>,    \
                                              C<T>*, int, const int*,           \
                                              cudaStream_t);                    \
  template void launch_resid_restrict<T, C<T>, C<T>, C<T>>(                     \
      const LevelDev&, const LevelDev&, int, Shift, VRef<T>, const C<T>*,       \
      C<T>*, int, const int*, cudaStream_t);                                    \
  template void launch_prolong_add<T, C<T>, C<T>>(const LevelDev&,              \
                                                  const LevelDev&, int,         \
                                                  const C<T>*, C<T>*, int,      \
                                                  const int*, cudaStream_t);    \
  template void launch_smooth<T, C<T>, C<T>, C<T>>(const LevelDev&, int, Shift, \
                                                   VRef<T>, const C<T>*, C<T>*, \
                                                   int, const int*,             \
                                                   cudaStream_t);               \
  template void launch_dense_mv<T, C<T>, C<T>>(int, const C<T>*, VRef<T>,       \
                                               C<T>*, int, const int*,          \
                                               cudaStream_t);

HZ_VC_SAME(double)
HZ_VC_SAME(float)

using bf2 = __nv_bfloat162;
template void launch_jacobi0<float, float2, bf2>(const LevelDev&, int, VRefE<float2>,
                                                 bf2*, int, const int*, cudaStream_t);
template void launch_jacobi0<float, bf2, bf2>(const LevelDev&, int, VRefE<bf2>, bf2*,
                                              int, const int*, cudaStream_t);
template void launch_resid_restrict<float, float2, bf2, bf2>(
    const LevelDev&, const LevelDev&, int, Shift, VRefE<float2>, const bf2*, bf2*, int,
    const int*, cudaStream_t);
template void launch_resid_restrict<float, bf2, bf2, bf2>(
    const LevelDev&, const LevelDev&, int, Shift, VRefE<bf2>, const bf2*, bf2*, int,
    const int*, cudaStream_t);
template void launch_prolong_add<float, bf2, bf2>(const LevelDev&, const LevelDev&, int,
                                                  const bf2*, bf2*, int, const int*,
                                                  cudaStream_t);
template void launch_smooth<float, float2, bf2, float2>(const LevelDev&, int, Shift,
                                                        VRefE<float2>, const bf2*,
                                                        float2*, int, const int*,
                                                        cudaStream_t);
template void launch_smooth<float, bf2, bf2, bf2>(const LevelDev&, int, Shift,
                                                  VRefE<bf2>, const bf2*, bf2*, int,
                                                  const int*, cudaStream_t);
template void launch_dense_mv<float, bf2, bf2>(int, const float2*, VRefE<bf2>, bf2*, int,
                                               const int*, cudaStream_t);

#define HZ_VC_FUSED(T, SF, SX, SC, SO)                                          \
  template void launch_pre_restrict<T, SF, SX, SC>(                             \
      const LevelDev&, const LevelDev&, int, Shift, VRefE<SF>, SX*, SC*, int,   \
      const int*, cudaStream_t);                                                \
  template void launch_pre_restrict_mr<T, SF, SX, SC>(                          \
      const LevelDev&, const LevelDev&, int, double, VRefE<SF>, SX*, SC*, int,  \
      int, const int*, cudaStream_t, unsigned long long*, long long);           \
  template void launch_prolong_smooth_mr<T, SC, SX, SF, SO>(                    \
      const LevelDev&, const LevelDev&, int, double, const SC*, const SX*,      \
      VRefE<SF>, SO*, int, int, int, const int*, cudaStream_t,                  \
      unsigned long long*, long long);                                          \
  template void launch_prolong_smooth<T, SC, SX, SF, SO>(                       \
      const LevelDev&, const LevelDev&, int, Shift, const SC*, const SX*,       \
      VRefE<SF>, SO*, int, const int*, cudaStream_t);
HZ_VC_FUSED(double, double2, double2, double2, double2)
HZ_VC_FUSED(float, float2, float2, float2, float2)
HZ_VC_FUSED(float, float2, bf2, bf2, float2)
HZ_VC_FUSED(float, bf2, bf2, bf2, bf2)

// staged kernels whose top-level input is the FP16 inner basis
#define HZ_VC_STAGED_IN16(SL)                                                   \
  template void launch_pre_restrict_mr<float, __half2, SL, SL>(                 \
      const LevelDev&, const LevelDev&, int, double, VRefE<__half2>, SL*, SL*,  \
      int, int, const int*, cudaStream_t, unsigned long long*, long long);      \
  template void launch_prolong_smooth_mr<float, SL, SL, __half2, float2>(       \
      const LevelDev&, const LevelDev&, int, double, const SL*, const SL*,      \
      VRefE<__half2>, float2*, int, int, int, const int*, cudaStream_t,         \
      unsigned long long*, long long);
HZ_VC_STAGED_IN16(float2)
HZ_VC_STAGED_IN16(bf2)

}  // namespace hz
