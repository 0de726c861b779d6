// Matrix-free grid kernels: Helmholtz / CSLP stencils (Sec. 2.1, 3.1, 5.1),
// damped Jacobi, full-weighting restriction and bilinear interpolation
// (Sec. 3.1, 3.2.1), higher-order deflation transfers (Sec. 3.2.1), the
// ReD-Glk coarse stencils (Sec. 5.2.4), the dense coarsest-level solve and
// the setup kernels.  Every kernel serves nrhs right-hand sides (blockIdx.z)
// and skips those flagged done.
#include <mutex>

#include "hz_common.cuh"
#include "hz_stencil_dev.cuh"

namespace hz {

namespace {

constexpr int BX = 32, BY = 8;

inline dim3 grid2d(int nx, int ny, int nrhs) {
  return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, nrhs);
}

template <class T>
__global__ void k_helm(LevelDev L, int bc, T sre, T sim, VRef<T> xin,
                       VRef<T> bin, C<T>* __restrict__ y,
                       const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || (done && done[r])) return;
  const long long n = (long long)L.nx * L.ny, id = (long long)j * L.nx + i;
  C<T>* yr = y + r * n;
  if (bc == BC_DIRICHLET && on_bnd(i, j, L.nx, L.ny)) {
    yr[id] = czero<T>();
    return;
  }
  const C<T> v = helm_point<T>(L, bc, sre, sim, xin.get() + r * n, i, j);
  yr[id] = bin.base ? bin.get()[r * n + id] - v : v;
}

// 1-D weights of Z^T: bilinear [1 2 1]/2 at offsets -1..1, higher-order
// [1 4 6 4 1]/8 at offsets -2..2; R_Z = Z^T / 4 is their tensor product / 4.
template <class T>
__global__ void k_restrict_z(LevelDev Lf, LevelDev Lc, int bc, int zk,
                             VRef<T> fin, C<T>* __restrict__ coarse,
                             const int* __restrict__ done, T scale) {
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (I >= Lc.nx || J >= Lc.ny || (done && done[r])) return;
  const long long nf = (long long)Lf.nx * Lf.ny, nc = (long long)Lc.nx * Lc.ny;
  const long long idc = (long long)J * Lc.nx + I;
  if (bc == BC_DIRICHLET && on_bnd(I, J, Lc.nx, Lc.ny)) {
    coarse[r * nc + idc] = czero<T>();
    return;
  }
  const C<T>* f = fin.get() + r * nf;
  const int rad = (zk == ZK_HO) ? 2 : 1;
  const T wb[3] = {T(0.5), T(1), T(0.5)};
  const T wh[5] = {T(0.125), T(0.5), T(0.75), T(0.5), T(0.125)};
  C<T> acc = czero<T>();
  for (int b = -rad; b <= rad; ++b) {
    const int jf = 2 * J + b;
    if (jf < 0 || jf >= Lf.ny) continue;
    const T wy = (zk == ZK_HO) ? wh[b + 2] : wb[b + 1];
    for (int a = -rad; a <= rad; ++a) {
      const int ifn = 2 * I + a;
      if (ifn < 0 || ifn >= Lf.nx) continue;
      if (bc == BC_DIRICHLET && on_bnd(ifn, jf, Lf.nx, Lf.ny)) continue;
      const T wx = (zk == ZK_HO) ? wh[a + 2] : wb[a + 1];
      acc = rfma(wx * wy * T(0.25), f[(long long)jf * Lf.nx + ifn], acc);
    }
  }
  coarse[r * nc + idc] = scale * acc;
}

// Z x at fine node (i, j): the three taps of each dimension at coarse base
// k, k+1, k+2 (ztaps below: weights 0 for the taps a rule does not use;
// higher-order taps outside the coarse grid are dropped), unrolled so that
// the taps stay in registers.
template <class T>
__device__ __forceinline__ int ztaps(int zk, int g, T& w0, T& w1, T& w2);

template <class T>
__global__ void k_prolong_z(LevelDev Lf, LevelDev Lc, int bc, int zk,
                            const C<T>* __restrict__ coarse,
                            C<T>* __restrict__ fine, int add,
                            const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= Lf.nx || j >= Lf.ny || (done && done[r])) return;
  const long long nf = (long long)Lf.nx * Lf.ny, nc = (long long)Lc.nx * Lc.ny;
  const long long id = (long long)j * Lf.nx + i;
  if (bc == BC_DIRICHLET && on_bnd(i, j, Lf.nx, Lf.ny)) {
    if (!add) fine[r * nf + id] = czero<T>();
    return;
  }
  T wx[3], wy[3];
  const int kx = ztaps<T>(zk, i, wx[0], wx[1], wx[2]);
  const int ky = ztaps<T>(zk, j, wy[0], wy[1], wy[2]);
  const C<T>* c = coarse + r * nc;
  C<T> acc = czero<T>();
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int cj = ky + b;
    if (wy[b] == T(0) || cj < 0 || cj >= Lc.ny) continue;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ci = kx + a;
      if (wx[a] == T(0) || ci < 0 || ci >= Lc.nx) continue;
      if (bc == BC_DIRICHLET && on_bnd(ci, cj, Lc.nx, Lc.ny)) continue;
      acc = rfma(wx[a] * wy[b], c[(long long)cj * Lc.nx + ci], acc);
    }
  }
  fine[r * nf + id] = add ? fine[r * nf + id] + acc : acc;
}

// str-Glk fused (Sec. 5.2.1): y = R_Z A_h Z x for a TC x TC tile of coarse
// outputs in one CTA.  The coarse tile with a halo of 2, the interpolated
// fine values Z x on the 2TC+5 square around it and A_h Z x on the 2TC+3
// square stay in shared memory, so each launch reads x and k^2 once and
// writes y once (the three-kernel form moves two fine-grid vectors through
// HBM twice).  Same boundary rules as k_prolong_z / k_helm / k_restrict_z.
// Interpolation taps of a fine index g along one dimension: the values at
// coarse base, base+1, base+2 get weights w0, w1, w2 (Z = bilinear or the
// higher-order rule; odd g lies between two coarse nodes).
template <class T>
__device__ __forceinline__ int ztaps(int zk, int g, T& w0, T& w1, T& w2) {
  const int K = g >> 1;  // floor(g / 2), also for negative g
  if (g & 1) {
    w0 = T(0.5); w1 = T(0.5); w2 = T(0);
    return K;
  }
  if (zk == ZK_HO) {
    w0 = T(0.125); w1 = T(0.75); w2 = T(0.125);
  } else {
    w0 = T(0); w1 = T(1); w2 = T(0);
  }
  return K - 1;
}

// Weight of fine offset a in the restriction R_Z = Z^T / 4 along one
// dimension (the 1/4 applied once at the end).
template <class T>
__device__ __forceinline__ T rtap(int zk, int a) {
  if (zk == ZK_HO) {
    switch (a) {
      case -2: case 2: return T(0.125);
      case -1: case 1: return T(0.5);
      default: return T(0.75);
    }
  }
  return (a == 0) ? T(1) : ((a == 1 || a == -1) ? T(0.5) : T(0));
}

// The interpolation and the restriction are tensor products of 1-D rules,
// so they run as an x pass then a y pass (3 + 3 taps instead of 9, 5 + 5
// instead of 25).  Shared buffers are reused between passes:
//   xs: coarse tile;  bufA: x-interpolated rows, then A z;
//   bufZ: z = Z x, then the x-restricted rows.
template <class T, int TC, int ZK>
__global__ void __launch_bounds__(TC * TC)
k_galerkin_fused(LevelDev Lf, LevelDev Lc, int bc, const C<T>* __restrict__ x,
                 C<T>* __restrict__ y, const int* __restrict__ done) {
  constexpr int CX = TC + 5, FZ = 2 * TC + 5, FA = 2 * TC + 3;
  __shared__ C<T> xs[CX * CX];
  __shared__ C<T> bufZ[FZ * FZ];
  __shared__ C<T> bufA[FA * FA];
  static_assert(CX * FZ <= FA * FA && FA * TC <= FZ * FZ, "buffer reuse");
  const int r = blockIdx.z;
  if (done && done[r]) return;
  const int I0 = blockIdx.x * TC, J0 = blockIdx.y * TC;
  const int nfx = Lf.nx, nfy = Lf.ny, ncx = Lc.nx, ncy = Lc.ny;
  const long long nc = (long long)ncx * ncy;
  const C<T>* xr = x + r * nc;
  const int tid = threadIdx.x, nt = TC * TC;
  // 1. coarse tile [I0-2, I0+TC+2]^2 (zero outside the grid and on
  //    Dirichlet boundary nodes, so Z is truncated there)
  for (int q = tid; q < CX * CX; q += nt) {
    const int ci = I0 - 2 + q % CX, cj = J0 - 2 + q / CX;
    C<T> v = czero<T>();
    if (ci >= 0 && ci < ncx && cj >= 0 && cj < ncy &&
        !(bc == BC_DIRICHLET && on_bnd(ci, cj, ncx, ncy)))
      v = xr[(long long)cj * ncx + ci];
    xs[q] = v;
  }
  __syncthreads();
  // 2a. interpolate along x: coarse rows x fine columns [2I0-3, 2I0+2TC+1]
  C<T>* zx = bufA;
  for (int q = tid; q < CX * FZ; q += nt) {
    const int cj = q / FZ, fi = q % FZ;
    T w0, w1, w2;
    const int bx = ztaps<T>(ZK, 2 * I0 - 3 + fi, w0, w1, w2) - (I0 - 2);
    const C<T>* row = xs + cj * CX + bx;
    zx[q] = rfma(w2, row[2], rfma(w1, row[1], w0 * row[0]));
  }
  __syncthreads();
  // 2b. interpolate along y: z on fine nodes [2I0-3, 2I0+2TC+1]^2, zero
  //     outside the grid and on Dirichlet boundary nodes
  for (int q = tid; q < FZ * FZ; q += nt) {
    const int fj = q / FZ, fi = q % FZ;
    const int gi = 2 * I0 - 3 + fi, gj = 2 * J0 - 3 + fj;
    C<T> v = czero<T>();
    if (gi >= 0 && gi < nfx && gj >= 0 && gj < nfy &&
        !(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy))) {
      T w0, w1, w2;
      const int by = ztaps<T>(ZK, gj, w0, w1, w2) - (J0 - 2);
      const C<T>* col = zx + by * FZ + fi;
      v = rfma(w2, col[2 * FZ], rfma(w1, col[FZ], w0 * col[0]));
    }
    bufZ[q] = v;
  }
  __syncthreads();
  // 3. A_h z on fine nodes [2I0-2, 2I0+2TC]^2
  const C<T>* zs = bufZ;
  C<T>* as = bufA;
  const T ih2 = ih2_of<T>(Lf);
  const T* k2 = k2_of<T>(Lf);
  for (int q = tid; q < FA * FA; q += nt) {
    const int ai = q % FA, aj = q / FA;
    const int gi = 2 * I0 - 2 + ai, gj = 2 * J0 - 2 + aj;
    C<T> v = czero<T>();
    if (gi >= 0 && gi < nfx && gj >= 0 && gj < nfy &&
        !(bc == BC_DIRICHLET && on_bnd(gi, gj, nfx, nfy))) {
      const T kk = k2[(long long)gj * nfx + gi];
      C<T> cen = mkc(T(4) * ih2 - kk, T(0));
      T cw = -ih2, ce = -ih2, cs = -ih2, cn = -ih2;
      if (bc == BC_SOMMERFELD) {
        const bool x0 = gi == 0, x1 = gi == nfx - 1, y0 = gj == 0, y1 = gj == nfy - 1;
        const int ns = int(x0) + int(x1) + int(y0) + int(y1);
        if (ns) {
          cen.y -= T(ns) * tih_of<T>(Lf) * sqrt(kk);
          if (x0) { cw = T(0); ce = T(2) * ce; }
          if (x1) { ce = T(0); cw = T(2) * cw; }
          if (y0) { cs = T(0); cn = T(2) * cn; }
          if (y1) { cn = T(0); cs = T(2) * cs; }
        }
      } else {
        if (gi == 1) cw = T(0);
        if (gi == nfx - 2) ce = T(0);
        if (gj == 1) cs = T(0);
        if (gj == nfy - 2) cn = T(0);
      }
      const int zc = (aj + 1) * FZ + (ai + 1);
      v = cmul(cen, zs[zc]);
      v = rfma(cw, zs[zc - 1], v);
      v = rfma(ce, zs[zc + 1], v);
      v = rfma(cs, zs[zc - FZ], v);
      v = rfma(cn, zs[zc + FZ], v);
    }
    as[q] = v;
  }
  __syncthreads();
  // 4a. restrict along x: fine rows [2J0-2, 2J0+2TC] x the tile's columns;
  //     fine nodes outside the grid hold zero in `as`
  C<T>* rx = bufZ;
  for (int q = tid; q < FA * TC; q += nt) {
    const int fa = q / TC, ti = q % TC;
    const C<T>* row = as + fa * FA + 2 * ti;
    C<T> v = czero<T>();
#pragma unroll
    for (int a = 0; a < 5; ++a) v = rfma(rtap<T>(ZK, a - 2), row[a], v);
    rx[q] = v;
  }
  __syncthreads();
  // 4b. restrict along y and scale by 1/4 (R_Z = Z^T / 4)
  const int ti = tid % TC, tj = tid / TC;
  const int I = I0 + ti, J = J0 + tj;
  if (I >= ncx || J >= ncy) return;
  C<T> acc = czero<T>();
  if (!(bc == BC_DIRICHLET && on_bnd(I, J, ncx, ncy))) {
    const C<T>* col = rx + (2 * tj) * TC + ti;
#pragma unroll
    for (int b = 0; b < 5; ++b) acc = rfma(rtap<T>(ZK, b - 2), col[b * TC], acc);
    acc = T(0.25) * acc;
  }
  y[r * nc + (long long)J * ncx + I] = acc;
}

// ReD-Glk (Sec. 5.2.4): printed 5x5 Galerkin Laplacian (scale 1/(256 H^2))
// and constant-k mass stencil (scale k^2/64^2), both divided by 4 so that
// the operator matches R = Z^T/4.  Rows: y offset -2..2, cols: x offset.
__constant__ float c_glk_lap[25] = {
    -3, -44, -98, -44, -3, -44, -112, 56, -112, -44, -98, 56, 980,
    56, -98, -44, -112, 56, -112, -44, -3, -44, -98, -44, -3};
__constant__ float c_glk_mass[25] = {
    1, 28, 70, 28, 1, 28, 784, 1960, 784, 28, 70, 1960, 4900,
    1960, 70, 28, 784, 1960, 784, 28, 1, 28, 70, 28, 1};

// Value of x at a node one layer outside the grid (ghost), Sec. 5.2.4:
// Sommerfeld u_g = u_in + 2 i H k_b u_b (eq. GhostPoint), Dirichlet
// u_g = 2 u_b - u_in with u_b = 0 (eq. DirchletGhostPoint).  Corner ghosts:
// the average of reaching them through x first (the rule along the ghost
// row) and through y first (along the ghost column).  That second
// application's boundary node is a ghost; the boundary condition holds on
// the boundary line continued past the corner, so it takes the wavenumber
// of the corner node.  (The zero wavenumber of ghost nodes belongs to the
// mass stencil only; here it would leave the corner rows inconsistent.)
template <class T>
__device__ C<T> glk_node(const LevelDev& L, int bc, const C<T>* __restrict__ x,
                         int i, int j) {
  const int nx = L.nx, ny = L.ny;
  const bool gx = (i < 0 || i >= nx), gy = (j < 0 || j >= ny);
  if (!gx && !gy) {
    if (bc == BC_DIRICHLET && on_bnd(i, j, nx, ny)) return czero<T>();
    return x[(long long)j * nx + i];
  }
  const T H2 = T(2) * T(L.h);
  const T* k2 = k2_of<T>(L);
  // real value at a node (Dirichlet boundary nodes are zero)
  auto val = [&](int a, int b) -> C<T> {
    if (bc == BC_DIRICHLET && on_bnd(a, b, nx, ny)) return czero<T>();
    return x[(long long)b * nx + a];
  };
  // ghost across x on real row b
  auto gxv = [&](int a, int b) -> C<T> {
    const int bi = (a < 0) ? 0 : nx - 1, ii = (a < 0) ? 1 : nx - 2;
    const C<T> ub = val(bi, b), ui = val(ii, b);
    if (bc == BC_SOMMERFELD) {
      const T kb = sqrt(k2[(long long)b * nx + bi]);
      return mkc(ui.x - H2 * kb * ub.y, ui.y + H2 * kb * ub.x);
    }
    return T(2) * ub - ui;
  };
  auto gyv = [&](int a, int b) -> C<T> {
    const int bj = (b < 0) ? 0 : ny - 1, jj = (b < 0) ? 1 : ny - 2;
    const C<T> ub = val(a, bj), ui = val(a, jj);
    if (bc == BC_SOMMERFELD) {
      const T kb = sqrt(k2[(long long)bj * nx + a]);
      return mkc(ui.x - H2 * kb * ub.y, ui.y + H2 * kb * ub.x);
    }
    return T(2) * ub - ui;
  };
  if (gx && !gy) return gxv(i, j);
  if (gy && !gx) return gyv(i, j);
  // corner ghost
  const int bi = (i < 0) ? 0 : nx - 1, ii = (i < 0) ? 1 : nx - 2;
  const int bj = (j < 0) ? 0 : ny - 1, jj = (j < 0) ? 1 : ny - 2;
  C<T> ox, oy;
  if (bc == BC_SOMMERFELD) {
    const T kc = sqrt(k2[(long long)bj * nx + bi]);
    const C<T> bx = gyv(bi, j), by = gxv(i, bj), ix = gyv(ii, j), iy = gxv(i, jj);
    ox = mkc(ix.x - H2 * kc * bx.y, ix.y + H2 * kc * bx.x);
    oy = mkc(iy.x - H2 * kc * by.y, iy.y + H2 * kc * by.x);
  } else {
    ox = T(2) * gyv(bi, j) - gyv(ii, j);
    oy = T(2) * gxv(i, bj) - gxv(i, jj);
  }
  return T(0.5) * (ox + oy);
}

template <class T>
__global__ void k_glk(LevelDev L, int bc, int variant, const C<T>* __restrict__ x,
                      C<T>* __restrict__ y, const int* __restrict__ done, T gscale) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || (done && done[r])) return;
  const int nx = L.nx, ny = L.ny;
  const long long n = (long long)nx * ny, id = (long long)j * nx + i;
  if (bc == BC_DIRICHLET && on_bnd(i, j, nx, ny)) {
    y[r * n + id] = czero<T>();
    return;
  }
  const C<T>* xr = x + r * n;
  const int dist = min(min(i, nx - 1 - i), min(j, ny - 1 - j));
  if (dist <= (variant == 2 ? 0 : 1)) {
    y[r * n + id] = helm_point<T>(L, bc, T(1), T(0), xr, i, j);
    return;
  }
  const T lap_s = ih2_of<T>(L) * T(1.0 / 1024.0);
  const T mass_s = T(1.0 / 16384.0);
  const T* k2 = k2_of<T>(L);
  C<T> acc = czero<T>();
  for (int dy = -2; dy <= 2; ++dy) {
    const int jn = j + dy;
    for (int dx = -2; dx <= 2; ++dx) {
      const int in = i + dx;
      const bool inside = in >= 0 && in < nx && jn >= 0 && jn < ny;
      const T k2n = inside ? k2[(long long)jn * nx + in] : T(0);
      const int s = (dy + 2) * 5 + (dx + 2);
      const T c = T(c_glk_lap[s]) * lap_s - T(c_glk_mass[s]) * mass_s * k2n;
      acc = rfma(c, glk_node<T>(L, bc, xr, in, jn), acc);
    }
  }
  y[r * n + id] = gscale * acc;
}

// ReD-O4 (Sec. 5.2.3): nodes whose 4th-order cross stays inside the grid use
// eq. (Helmstencil Oh4), -[-1 16 -30 16 -1] / (12 H^2) along x and y minus
// k^2 of the node; nodes within one node of the boundary use the ReD-O2 row.
// Dirichlet boundary nodes hold zero (their values in x are not read).
template <class T>
__global__ void k_red_o4(LevelDev L, int bc, const C<T>* __restrict__ x,
                         C<T>* __restrict__ y, const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || (done && done[r])) return;
  const int nx = L.nx, ny = L.ny;
  const long long n = (long long)nx * ny, id = (long long)j * nx + i;
  const C<T>* xr = x + r * n;
  if (bc == BC_DIRICHLET && on_bnd(i, j, nx, ny)) {
    y[r * n + id] = czero<T>();
    return;
  }
  const int dist = min(min(i, nx - 1 - i), min(j, ny - 1 - j));
  if (dist <= 1) {
    y[r * n + id] = helm_point<T>(L, bc, T(1), T(0), xr, i, j);
    return;
  }
  auto xv = [&](int a, int b) {
    if (bc == BC_DIRICHLET && on_bnd(a, b, nx, ny)) return czero<T>();
    return xr[(long long)b * nx + a];
  };
  const T s = ih2_of<T>(L) / T(12);
  const T k2 = k2_of<T>(L)[id];
  C<T> acc = (T(60) * s - k2) * xr[id];
  acc = rfma(T(-16) * s, (xv(i - 1, j) + xv(i + 1, j)) + (xv(i, j - 1) + xv(i, j + 1)), acc);
  acc = rfma(s, (xv(i - 2, j) + xv(i + 2, j)) + (xv(i, j - 2) + xv(i, j + 2)), acc);
  y[r * n + id] = acc;
}

// ReD-O6 (Sec. 5.2.3): the sixth-order cross (2 -27 270 -490 270 -27 2) /
// (180 H^2) along x and y, negated, minus k^2 of the node, where the cross
// stays inside the grid; nodes within two nodes of the boundary use ReD-O2.
template <class T>
__global__ void k_red_o6(LevelDev L, int bc, const C<T>* __restrict__ x,
                         C<T>* __restrict__ y, const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || (done && done[r])) return;
  const int nx = L.nx, ny = L.ny;
  const long long n = (long long)nx * ny, id = (long long)j * nx + i;
  const C<T>* xr = x + r * n;
  if (bc == BC_DIRICHLET && on_bnd(i, j, nx, ny)) {
    y[r * n + id] = czero<T>();
    return;
  }
  if (min(min(i, nx - 1 - i), min(j, ny - 1 - j)) <= 2) {
    y[r * n + id] = helm_point<T>(L, bc, T(1), T(0), xr, i, j);
    return;
  }
  auto xv = [&](int a, int b) {
    if (bc == BC_DIRICHLET && on_bnd(a, b, nx, ny)) return czero<T>();
    return xr[(long long)b * nx + a];
  };
  const T s = ih2_of<T>(L) / T(180);
  const T k2 = k2_of<T>(L)[id];
  C<T> acc = (T(980) * s - k2) * xr[id];
  acc = rfma(T(-270) * s, (xv(i - 1, j) + xv(i + 1, j)) + (xv(i, j - 1) + xv(i, j + 1)), acc);
  acc = rfma(T(27) * s, (xv(i - 2, j) + xv(i + 2, j)) + (xv(i, j - 2) + xv(i, j + 2)), acc);
  acc = rfma(T(-2) * s, (xv(i - 3, j) + xv(i + 3, j)) + (xv(i, j - 3) + xv(i, j + 3)), acc);
  y[r * n + id] = acc;
}

// ReD-cmpO4 (Sec. 5.2.5): the compact 3x3 stencil [a] / H^2 - [b] k^2 of
// eq. (GeneralFormReD) with the Singer-Turkel weights (gamma = 1), each
// mass entry with its own node's k^2.  Under Sommerfeld rows the ghost
// layer is u_g = 2 i k H (1 - k^2 H^2 / 6) u_b + u_in (k of the boundary
// node, ghost k^2 = 0), a corner ghost the average of its two neighbouring
// edge ghosts; Dirichlet boundary nodes hold zero.
// The same kernel serves ReD-9ptO2 (Appendix B; SCHEME 1): a = (4.632,
// -1.316, 0.158), b = (1, 0, 0), with the 2nd-order ghost rule of eq.
// (GhostPoint), u_g = 2 i k H u_b + u_in.
template <class T, int SCHEME>
__device__ __forceinline__ C<T> cmp_edge_ghost(const LevelDev& L, const C<T>* xr, int bi,
                                               int bj, int ii, int ij) {
  const long long b = (long long)bj * L.nx + bi;
  const T k = sqrt(k2_of<T>(L)[b]);
  const T H = T(L.h);
  const T c = SCHEME == 0 ? T(2) * k * H * (T(1) - k * k * H * H / T(6)) : T(2) * k * H;
  const C<T> ub = xr[b];
  return mkc(-c * ub.y, c * ub.x) + xr[(long long)ij * L.nx + ii];
}
template <class T, int SCHEME>
__device__ __forceinline__ C<T> cmp_node(const LevelDev& L, int bc, const C<T>* xr,
                                         int i, int j) {
  const int nx = L.nx, ny = L.ny;
  const bool gx = i < 0 || i >= nx, gy = j < 0 || j >= ny;
  if (!gx && !gy) {
    if (bc == BC_DIRICHLET && on_bnd(i, j, nx, ny)) return czero<T>();
    return xr[(long long)j * nx + i];
  }
  // ghosts exist only under Sommerfeld rows (Dirichlet rows never reach them)
  const int bi = i < 0 ? 0 : (i >= nx ? nx - 1 : i);
  const int bj = j < 0 ? 0 : (j >= ny ? ny - 1 : j);
  const int ii = i < 0 ? 1 : (i >= nx ? nx - 2 : i);
  const int ij = j < 0 ? 1 : (j >= ny ? ny - 2 : j);
  if (gx && !gy) return cmp_edge_ghost<T, SCHEME>(L, xr, bi, j, ii, j);
  if (!gx && gy) return cmp_edge_ghost<T, SCHEME>(L, xr, i, bj, i, ij);
  // corner: average of the y ghost of (bi, .) and the x ghost of (., bj)
  return T(0.5) * (cmp_edge_ghost<T, SCHEME>(L, xr, bi, bj, bi, ij) +
                   cmp_edge_ghost<T, SCHEME>(L, xr, bi, bj, ii, bj));
}
template <class T, int SCHEME>
__global__ void k_red_cmpo4(LevelDev L, int bc, const C<T>* __restrict__ x,
                            C<T>* __restrict__ y, const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || (done && done[r])) return;
  const int nx = L.nx, ny = L.ny;
  const long long n = (long long)nx * ny, id = (long long)j * nx + i;
  const C<T>* xr = x + r * n;
  if (bc == BC_DIRICHLET && on_bnd(i, j, nx, ny)) {
    y[r * n + id] = czero<T>();
    return;
  }
  const T ih2 = ih2_of<T>(L);
  const T* k2 = k2_of<T>(L);
  const T a0 = SCHEME == 0 ? T(10) / T(3) : T(4.632);
  const T as = SCHEME == 0 ? T(-2) / T(3) : T(-1.316);
  const T ac = SCHEME == 0 ? T(-1) / T(6) : T(0.158);
  const T b0 = SCHEME == 0 ? T(2) / T(3) + T(1) / T(36) : T(1);
  const T bs = SCHEME == 0 ? T(1) / T(12) - T(1) / T(72) : T(0);
  const T bc_ = SCHEME == 0 ? T(1) / T(144) : T(0);
  C<T> acc = czero<T>();
  for (int dj = -1; dj <= 1; ++dj)
    for (int di = -1; di <= 1; ++di) {
      const int a = i + di, b = j + dj;
      const bool in = a >= 0 && a < nx && b >= 0 && b < ny;
      const T kk = in ? k2[(long long)b * nx + a] : T(0);
      const int d = abs(di) + abs(dj);
      const T wa = d == 0 ? a0 : (d == 1 ? as : ac);
      const T wb = d == 0 ? b0 : (d == 1 ? bs : bc_);
      acc = rfma(wa * ih2 - wb * kk, cmp_node<T, SCHEME>(L, bc, xr, a, b), acc);
    }
  y[r * n + id] = acc;
}

template <class T>
__global__ void k_mask_dirichlet(LevelDev L, C<T>* __restrict__ x) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || !on_bnd(i, j, L.nx, L.ny)) return;
  x[(long long)r * L.nx * L.ny + (long long)j * L.nx + i] = czero<T>();
}

template <class T> __device__ __forceinline__ C<T> cvt(double2 v);
template <> __device__ __forceinline__ double2 cvt<double>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt<float>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}
template <class T> __device__ __forceinline__ double2 widen(C<T> v);
template <> __device__ __forceinline__ double2 widen<double>(double2 v) { return v; }
template <> __device__ __forceinline__ double2 widen<float>(float2 v) {
  return make_double2(v.x, v.y);
}

// ---------------------------------------------------------------------------
// stcl-op-Glk (Sec. 5.2.1, Table 1): the Galerkin operator E = R_Z A_h Z
// stored as one (2R+1) x (2R+1) stencil per coarse node (R = 2 for the
// higher-order Z, 1 for bilinear Z) and applied as a stencil.  The
// coefficients are extracted at setup by applying the on-the-fly product to
// P^2 probe vectors (P = 2R+1), probe c = (cx, cy) holding 1 on the coarse
// nodes J with J mod P = c: since E couples nodes at most R apart, (E p_c)(I)
// is the single coefficient E(I, J) of the J of probe c within R of I.

// out[b] = probe c0 + b (FP64), b < nprobe
__global__ void k_probe_fill(LevelDev Lc, int P, int c0, double2* __restrict__ out) {
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y;
  const int b = blockIdx.z;
  if (I >= Lc.nx || J >= Lc.ny) return;
  const int c = c0 + b, cx = c % P, cy = c / P;
  const long long nc = (long long)Lc.nx * Lc.ny;
  out[b * nc + (long long)J * Lc.nx + I] =
      make_double2((I % P == cx && J % P == cy) ? 1.0 : 0.0, 0.0);
}

// S[k][I] = (E p_c)(I) for the stencil slot k of the offset from I to the
// probe node of c; S holds (2R+1)^2 coefficient planes of nc values
template <class T>
__global__ void k_probe_extract(LevelDev Lc, int P, int c0,
                                const double2* __restrict__ ep, C<T>* __restrict__ S) {
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y;
  const int b = blockIdx.z;
  if (I >= Lc.nx || J >= Lc.ny) return;
  const int R = P / 2, c = c0 + b, cx = c % P, cy = c / P;
  int dx = ((cx - I) % P + P) % P, dy = ((cy - J) % P + P) % P;
  if (dx > R) dx -= P;
  if (dy > R) dy -= P;
  const long long nc = (long long)Lc.nx * Lc.ny, id = (long long)J * Lc.nx + I;
  S[(long long)((dy + R) * P + (dx + R)) * nc + id] = cvt<T>(ep[b * nc + id]);
}

// y = E x with the stored stencil; one thread per coarse node keeps its
// coefficients in registers while the block walks over its right-hand sides
// (blockIdx.z selects a group of rpb of them).  Each right-hand side's x
// tile with its halo is copied into a ring of NS shared-memory stages by
// cp.async, NS-1 right-hand sides ahead of the one being applied, so the
// DRAM bytes in flight per SM are set by the ring (the coefficients take
// the registers).
constexpr int kStencilNS = 6;

template <class T, int R>
struct StencilE {
  static constexpr int P = 2 * R + 1, K = P * P, TX = BX + 2 * R, TY = BY + 2 * R;
  static constexpr int NT = BX * BY, NPT = (TY * TX + NT - 1) / NT;
  static constexpr int STAGE = ((TY * TX * (int)sizeof(C<T>)) + 15) & ~15;
  static constexpr int smem(int rpb) { return kStencilNS * STAGE + 4 * rpb; }
};

template <class T, int R>
__global__ void __launch_bounds__(BX * BY)
k_stencil_e(LevelDev Lc, const C<T>* __restrict__ S, const C<T>* __restrict__ x,
            C<T>* __restrict__ y, int nrhs, int rpb, const int* __restrict__ done) {
  using Q = StencilE<T, R>;
  constexpr int P = Q::P, K = Q::K, TX = Q::TX, TY = Q::TY, NT = Q::NT, NPT = Q::NPT;
  constexpr int NS = kStencilNS, SV = Q::STAGE / (int)sizeof(C<T>);
  extern __shared__ __align__(16) unsigned char smraw[];
  C<T>* xs = reinterpret_cast<C<T>*>(smraw);
  int* act = reinterpret_cast<int*>(smraw + NS * Q::STAGE);
  __shared__ int nact_s;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int I0 = blockIdx.x * BX, J0 = blockIdx.y * BY;
  const int I = I0 + tx, J = J0 + ty;
  const int ncx = Lc.nx, ncy = Lc.ny;
  const long long nc = (long long)ncx * ncy;
  const bool in = I < ncx && J < ncy;
  const long long id = (long long)J * ncx + I;
  const int r0 = blockIdx.z * rpb, r1 = min(nrhs, r0 + rpb);
  // active right-hand sides of the group, listed by warp 0
  if (tid < 32) {
    int cnt = 0;
    for (int base = r0; base < r1; base += 32) {
      const int r = base + tid;
      const bool a = r < r1 && !(done && done[r]);
      const unsigned m = __ballot_sync(0xffffffffu, a);
      if (a) act[cnt + __popc(m & ((1u << tid) - 1u))] = r;
      cnt += __popc(m);
    }
    if (tid == 0) nact_s = cnt;
  }
  __syncthreads();
  const int na = nact_s;
  if (na == 0) return;
  C<T> cf[K];
#pragma unroll
  for (int k = 0; k < K; ++k) cf[k] = in ? S[(long long)k * nc + id] : czero<T>();
  // tile entries: node index, or -1 outside the grid (zero in every stage)
  int gid[NPT];
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    const int q = tid + u * NT;
    const int gi = I0 - R + q % TX, gj = J0 - R + q / TX;
    gid[u] = (q < TY * TX && gi >= 0 && gi < ncx && gj >= 0 && gj < ncy) ? gj * ncx + gi : -1;
    if (q < TY * TX && gid[u] < 0)
      for (int sidx = 0; sidx < NS; ++sidx) xs[sidx * SV + q] = czero<T>();
  }
  auto issue = [&](int k) {
    if (k < na) {
      const C<T>* xr = x + (long long)act[k] * nc;
      C<T>* stg = xs + (k % NS) * SV;
#pragma unroll
      for (int u = 0; u < NPT; ++u)
        if (gid[u] >= 0) cp_async_el<sizeof(C<T>)>(stg + tid + u * NT, xr + gid[u]);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) issue(k);
  for (int k = 0; k < na; ++k) {
    cp_async_wait<NS - 2>();
    __syncthreads();
    issue(k + NS - 1);
    if (in) {
      const C<T>* stg = xs + (k % NS) * SV;
      C<T> acc = czero<T>();
#pragma unroll
      for (int b = 0; b < P; ++b)
#pragma unroll
        for (int a = 0; a < P; ++a) acc = cfma(cf[b * P + a], stg[(ty + b) * TX + tx + a], acc);
      y[(long long)act[k] * nc + id] = acc;
    }
  }
  cp_async_wait<0>();
}


// The same product with each thread applying the stencil at two nodes of a
// column, (I, J) and (I, J + 1): the 2R + 2 rows of x it reads serve both
// (about 0.6 of the shared-memory loads per node of the one-node form), the
// block is BX x BY / 2 threads over the same BX x BY tile of nodes.
template <class T, int R>
__global__ void __launch_bounds__(BX * BY / 2, 4)
k_stencil_e2(LevelDev Lc, const C<T>* __restrict__ S, const C<T>* __restrict__ x,
             C<T>* __restrict__ y, int nrhs, int rpb, const int* __restrict__ done) {
  using Q = StencilE<T, R>;
  constexpr int P = Q::P, K = Q::K, TX = Q::TX, TY = Q::TY;
  constexpr int NT = BX * BY / 2, NPT = (TY * TX + NT - 1) / NT;
  constexpr int NS = kStencilNS, SV = Q::STAGE / (int)sizeof(C<T>);
  extern __shared__ __align__(16) unsigned char smraw[];
  C<T>* xs = reinterpret_cast<C<T>*>(smraw);
  int* act = reinterpret_cast<int*>(smraw + NS * Q::STAGE);
  __shared__ int nact_s;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int I0 = blockIdx.x * BX, J0 = blockIdx.y * BY;
  const int I = I0 + tx, J = J0 + 2 * ty;
  const int ncx = Lc.nx, ncy = Lc.ny;
  const long long nc = (long long)ncx * ncy;
  const bool in0 = I < ncx && J < ncy, in1 = I < ncx && J + 1 < ncy;
  const long long id = (long long)J * ncx + I;
  const int r0 = blockIdx.z * rpb, r1 = min(nrhs, r0 + rpb);
  if (tid < 32) {
    int cnt = 0;
    for (int base = r0; base < r1; base += 32) {
      const int r = base + tid;
      const bool a = r < r1 && !(done && done[r]);
      const unsigned m = __ballot_sync(0xffffffffu, a);
      if (a) act[cnt + __popc(m & ((1u << tid) - 1u))] = r;
      cnt += __popc(m);
    }
    if (tid == 0) nact_s = cnt;
  }
  __syncthreads();
  const int na = nact_s;
  if (na == 0) return;
  C<T> c0[K], c1[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    c0[k] = in0 ? S[(long long)k * nc + id] : czero<T>();
    c1[k] = in1 ? S[(long long)k * nc + id + ncx] : czero<T>();
  }
  int gid[NPT];
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    const int q = tid + u * NT;
    const int gi = I0 - R + q % TX, gj = J0 - R + q / TX;
    gid[u] = (q < TY * TX && gi >= 0 && gi < ncx && gj >= 0 && gj < ncy) ? gj * ncx + gi : -1;
    if (q < TY * TX && gid[u] < 0)
      for (int sidx = 0; sidx < NS; ++sidx) xs[sidx * SV + q] = czero<T>();
  }
  auto issue = [&](int k) {
    if (k < na) {
      const C<T>* xr = x + (long long)act[k] * nc;
      C<T>* stg = xs + (k % NS) * SV;
#pragma unroll
      for (int u = 0; u < NPT; ++u)
        if (gid[u] >= 0) cp_async_el<sizeof(C<T>)>(stg + tid + u * NT, xr + gid[u]);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) issue(k);
  for (int k = 0; k < na; ++k) {
    cp_async_wait<NS - 2>();
    __syncthreads();
    issue(k + NS - 1);
    const C<T>* stg = xs + (k % NS) * SV + (2 * ty) * TX + tx;
    C<T> a0 = czero<T>(), a1 = czero<T>();
#pragma unroll
    for (int b = 0; b <= P; ++b)
#pragma unroll
      for (int a = 0; a < P; ++a) {
        const C<T> v = stg[b * TX + a];
        if (b < P) a0 = cfma(c0[b * P + a], v, a0);
        if (b > 0) a1 = cfma(c1[(b - 1) * P + a], v, a1);
      }
    C<T>* yr = y + (long long)act[k] * nc + id;
    if (in0) yr[0] = a0;
    if (in1) yr[ncx] = a1;
  }
  cp_async_wait<0>();
}


template <class Ti, class To>
__global__ void k_add_conv(VRef<Ti> a, const C<Ti>* __restrict__ b, VRef<To> out,
                           long long n, const int* __restrict__ done) {
  const int r = blockIdx.y;
  if (done && done[r]) return;
  const C<Ti>* ar = a.get() + r * n;
  C<To>* orow = out.get() + r * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    C<Ti> v = ar[e];
    if (b) v = v + b[r * n + e];
    orow[e] = cvt<To>(widen<Ti>(v));
  }
}

// out = a - b (same precision)
template <class T>
__global__ void k_sub(const C<T>* __restrict__ a, const C<T>* __restrict__ b,
                      C<T>* __restrict__ out, long long n, const int* __restrict__ done) {
  const int r = blockIdx.y;
  if (done && done[r]) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[r * n + e] = a[r * n + e] - b[r * n + e];
}

// out = a - b + c in FP64 (the last step of the TLKM preconditioner)
template <class T>
__global__ void k_sub_add_widen(const C<T>* __restrict__ a, const C<T>* __restrict__ b,
                                const C<T>* __restrict__ c, VRef<double> out, long long n,
                                const int* __restrict__ done) {
  const int r = blockIdx.y;
  if (done && done[r]) return;
  double2* orow = out.get() + r * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long id = r * n + e;
    orow[e] = widen<T>((a[id] - b[id]) + c[id]);
  }
}

// ---------------------------------------------------------------- setup
__global__ void k_inject(LevelDev Lf, LevelDev Lc, double* k2c) {
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y;
  if (I >= Lc.nx || J >= Lc.ny) return;
  k2c[(long long)J * Lc.nx + I] = Lf.k2d[(long long)(2 * J) * Lf.nx + 2 * I];
}

__global__ void k_cast(const double* a, float* b, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    b[e] = (float)a[e];
}

// diagonal of M: 4/h^2 - (b1 + i b2) k^2 - i * sides * 2 k / h
__device__ __forceinline__ double2 diag_m(const LevelDev& L, int bc, Shift s,
                                          int i, int j) {
  const double k2 = L.k2d[(long long)j * L.nx + i];
  double2 d = make_double2(4.0 * L.ih2d - s.re * k2, -s.im * k2);
  if (bc == BC_SOMMERFELD) {
    const int ns = int(i == 0) + int(i == L.nx - 1) + int(j == 0) + int(j == L.ny - 1);
    d.y -= ns * L.tihd * sqrt(k2);
  }
  return d;
}

__global__ void k_dinv(LevelDev L, int bc, Shift s, double omega, double2* dd,
                       float2* df) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i >= L.nx || j >= L.ny) return;
  const long long id = (long long)j * L.nx + i;
  double2 v = make_double2(0.0, 0.0);
  if (!(bc == BC_DIRICHLET && on_bnd(i, j, L.nx, L.ny))) {
    const double2 d = diag_m(L, bc, s, i, j);
    const double m2 = d.x * d.x + d.y * d.y;
    v = make_double2(omega * d.x / m2, -omega * d.y / m2);
  }
  if (dd) dd[id] = v;
  if (df) df[id] = make_float2((float)v.x, (float)v.y);
}

// Row p of [M | I] (n x 2n) for the coarsest level; Dirichlet boundary rows
// are identity rows (those nodes carry zero).
__global__ void k_dense_assemble(LevelDev L, int bc, Shift s, double2* aug) {
  const int n = L.nx * L.ny;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double2* row = aug + (long long)p * 2 * n;
  for (int c = 0; c < 2 * n; ++c) row[c] = make_double2(0.0, 0.0);
  row[n + p] = make_double2(1.0, 0.0);
  const int i = p % L.nx, j = p / L.nx;
  if (bc == BC_DIRICHLET && on_bnd(i, j, L.nx, L.ny)) {
    row[p] = make_double2(1.0, 0.0);
    return;
  }
  row[p] = diag_m(L, bc, s, i, j);
  const double ih2 = L.ih2d;
  double cw = -ih2, ce = -ih2, cs = -ih2, cn = -ih2;
  if (bc == BC_SOMMERFELD) {
    if (i == 0) { cw = 0; ce *= 2; }
    if (i == L.nx - 1) { ce = 0; cw *= 2; }
    if (j == 0) { cs = 0; cn *= 2; }
    if (j == L.ny - 1) { cn = 0; cs *= 2; }
  } else {
    if (i == 1) cw = 0;
    if (i == L.nx - 2) ce = 0;
    if (j == 1) cs = 0;
    if (j == L.ny - 2) cn = 0;
  }
  if (cw != 0) row[p - 1] = make_double2(cw, 0.0);
  if (ce != 0) row[p + 1] = make_double2(ce, 0.0);
  if (cs != 0) row[p - L.nx] = make_double2(cs, 0.0);
  if (cn != 0) row[p + L.nx] = make_double2(cn, 0.0);
}

// Gauss-Jordan elimination with partial pivoting on [M | I] in one block.
__global__ void k_gauss_jordan(int n, double2* aug, int* err) {
  extern __shared__ unsigned char smraw[];
  double2* colk = reinterpret_cast<double2*>(smraw);   // n entries
  __shared__ double bestv[32];
  __shared__ int besti[32];
  __shared__ int piv;
  const int tid = threadIdx.x, nt = blockDim.x, w2 = 2 * n;
  for (int k = 0; k < n; ++k) {
    double bv = -1.0;
    int bi = k;
    for (int r = k + tid; r < n; r += nt) {
      const double2 a = aug[(long long)r * w2 + k];
      const double m = a.x * a.x + a.y * a.y;
      if (m > bv) { bv = m; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, bv, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv) { bv = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { bestv[tid >> 5] = bv; besti[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      double v = -1.0;
      int ix = k;
      for (int q = 0; q < (nt + 31) / 32; ++q)
        if (bestv[q] > v) { v = bestv[q]; ix = besti[q]; }
      piv = (v > 0.0) ? ix : -1;
      if (v <= 0.0) *err = 1;
    }
    __syncthreads();
    if (piv < 0) return;
    if (piv != k) {
      for (int c = tid; c < w2; c += nt) {
        const double2 t = aug[(long long)k * w2 + c];
        aug[(long long)k * w2 + c] = aug[(long long)piv * w2 + c];
        aug[(long long)piv * w2 + c] = t;
      }
    }
    __syncthreads();
    const double2 p = aug[(long long)k * w2 + k];
    const double pm = p.x * p.x + p.y * p.y;
    const double2 ip = make_double2(p.x / pm, -p.y / pm);
    __syncthreads();
    for (int c = tid; c < w2; c += nt) {
      const double2 a = aug[(long long)k * w2 + c];
      aug[(long long)k * w2 + c] =
          make_double2(a.x * ip.x - a.y * ip.y, a.x * ip.y + a.y * ip.x);
    }
    for (int r = tid; r < n; r += nt) colk[r] = aug[(long long)r * w2 + k];
    __syncthreads();
    for (long long e = tid; e < (long long)n * w2; e += nt) {
      const int r = (int)(e / w2), c = (int)(e % w2);
      if (r == k) continue;
      const double2 f = colk[r];
      if (f.x == 0.0 && f.y == 0.0) continue;
      const double2 a = aug[(long long)k * w2 + c];
      double2 t = aug[e];
      t.x -= f.x * a.x - f.y * a.y;
      t.y -= f.x * a.y + f.y * a.x;
      aug[e] = t;
    }
    __syncthreads();
  }
}

__global__ void k_extract(LevelDev L, int bc, const double2* aug, double2* md,
                          float2* mf) {
  const int n = L.nx * L.ny;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int r = (int)(e / n), c = (int)(e % n);
  double2 v = aug[(long long)r * 2 * n + n + c];
  if (bc == BC_DIRICHLET && (on_bnd(r % L.nx, r / L.nx, L.nx, L.ny) ||
                             on_bnd(c % L.nx, c / L.nx, L.nx, L.ny)))
    v = make_double2(0.0, 0.0);
  if (md) md[e] = v;
  if (mf) mf[e] = make_float2((float)v.x, (float)v.y);
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <class T>
void launch_helm(const LevelDev& L, int bc, Shift s, VRef<T> x, VRef<T> b,
                 C<T>* y, int nrhs, const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_helm<T><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(
      L, bc, (T)s.re, (T)s.im, x, b, y, done);
}
template <class T>
void launch_restrict_z(const LevelDev& Lf, const LevelDev& Lc, int bc, int zk,
                       VRef<T> fine, C<T>* coarse, int nrhs, const int* done,
                       cudaStream_t st, double scale) {
  HZ_COUNT();
  k_restrict_z<T><<<grid2d(Lc.nx, Lc.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, zk, fine, coarse, done, T(scale));
}
template <class T>
void launch_prolong_z(const LevelDev& Lf, const LevelDev& Lc, int bc, int zk,
                      const C<T>* coarse, C<T>* fine, int add, int nrhs,
                      const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_prolong_z<T><<<grid2d(Lf.nx, Lf.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, zk, coarse, fine, add, done);
}
template <class T>
void launch_galerkin_fused(const LevelDev& Lf, const LevelDev& Lc, int bc, int zk,
                           const C<T>* x, C<T>* y, int nrhs, const int* done,
                           cudaStream_t st) {
  HZ_COUNT();
  constexpr int TC = 16;
  const dim3 grid((Lc.nx + TC - 1) / TC, (Lc.ny + TC - 1) / TC, nrhs);
  if (zk == ZK_HO)
    k_galerkin_fused<T, TC, ZK_HO><<<grid, TC * TC, 0, st>>>(Lf, Lc, bc, x, y, done);
  else
    k_galerkin_fused<T, TC, ZK_BILINEAR><<<grid, TC * TC, 0, st>>>(Lf, Lc, bc, x, y, done);
}
void launch_probe_fill(const LevelDev& Lc, int P, int c0, int nprobe, double2* out,
                       cudaStream_t st) {
  HZ_COUNT();
  k_probe_fill<<<grid2d(Lc.nx, Lc.ny, nprobe), dim3(BX, BY), 0, st>>>(Lc, P, c0, out);
}
template <class T>
void launch_probe_extract(const LevelDev& Lc, int P, int c0, int nprobe,
                          const double2* ep, C<T>* S, cudaStream_t st) {
  HZ_COUNT();
  k_probe_extract<T><<<grid2d(Lc.nx, Lc.ny, nprobe), dim3(BX, BY), 0, st>>>(Lc, P, c0, ep,
                                                                          S);
}
template <class T>
void launch_stencil_e(const LevelDev& Lc, int R, int pairs, const C<T>* S, const C<T>* x,
                      C<T>* y, int nrhs, int rpb, const int* done, cudaStream_t st) {
  HZ_COUNT();
  if (rpb <= 0 || rpb > nrhs) rpb = nrhs;
  const dim3 grid((Lc.nx + BX - 1) / BX, (Lc.ny + BY - 1) / BY, (nrhs + rpb - 1) / rpb);
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute((const void*)k_stencil_e<T, 2>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         StencilE<T, 2>::smem(1024));
    cudaFuncSetAttribute((const void*)k_stencil_e<T, 1>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         StencilE<T, 1>::smem(1024));
    cudaFuncSetAttribute((const void*)k_stencil_e2<T, 2>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         StencilE<T, 2>::smem(1024));
    cudaFuncSetAttribute((const void*)k_stencil_e2<T, 1>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         StencilE<T, 1>::smem(1024));
  });
  if (pairs) {
    const dim3 blk(BX, BY / 2);
    if (R == 2)
      k_stencil_e2<T, 2><<<grid, blk, StencilE<T, 2>::smem(rpb), st>>>(Lc, S, x, y, nrhs,
                                                                      rpb, done);
    else
      k_stencil_e2<T, 1><<<grid, blk, StencilE<T, 1>::smem(rpb), st>>>(Lc, S, x, y, nrhs,
                                                                      rpb, done);
    return;
  }
  if (R == 2)
    k_stencil_e<T, 2><<<grid, dim3(BX, BY), StencilE<T, 2>::smem(rpb), st>>>(Lc, S, x, y,
                                                                           nrhs, rpb, done);
  else
    k_stencil_e<T, 1><<<grid, dim3(BX, BY), StencilE<T, 1>::smem(rpb), st>>>(Lc, S, x, y,
                                                                           nrhs, rpb, done);
}
template <class T>
void launch_glk(const LevelDev& L, int bc, int variant, const C<T>* x, C<T>* y,
                int nrhs, const int* done, cudaStream_t st, double gscale) {
  HZ_COUNT();
  k_glk<T><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(L, bc, variant, x,
                                                               y, done, T(gscale));
}
template <class T>
void launch_red_o4(const LevelDev& L, int bc, const C<T>* x, C<T>* y, int nrhs,
                   const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_red_o4<T><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(L, bc, x, y, done);
}
template <class T>
void launch_red_cmpo4(const LevelDev& L, int bc, const C<T>* x, C<T>* y, int nrhs,
                      const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_red_cmpo4<T, 0><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(L, bc, x, y, done);
}
template <class T>
void launch_red_9pt(const LevelDev& L, int bc, const C<T>* x, C<T>* y, int nrhs,
                    const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_red_cmpo4<T, 1><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(L, bc, x, y, done);
}
template <class T>
void launch_red_o6(const LevelDev& L, int bc, const C<T>* x, C<T>* y, int nrhs,
                   const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_red_o6<T><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(L, bc, x, y, done);
}
template <class T>
void launch_mask_dirichlet(const LevelDev& L, int bc, C<T>* x, int nrhs,
                           cudaStream_t st) {
  if (bc != BC_DIRICHLET) return;
  HZ_COUNT();
  k_mask_dirichlet<T><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(L, x);
}
template <class Ti, class To>
void launch_add_conv(VRef<Ti> a, const C<Ti>* b, VRef<To> out, long long n,
                     int nrhs, const int* done, cudaStream_t st) {
  HZ_COUNT();
  long long nb = (n + 255) / 256;
  if (nb > 4096) nb = 4096;
  k_add_conv<Ti, To><<<dim3((unsigned)nb, nrhs), 256, 0, st>>>(a, b, out, n, done);
}

template <class T>
void launch_sub(const C<T>* a, const C<T>* b, C<T>* out, long long n, int nrhs,
                const int* done, cudaStream_t st) {
  HZ_COUNT();
  long long nb = (n + 255) / 256;
  if (nb > 4096) nb = 4096;
  k_sub<T><<<dim3((unsigned)nb, nrhs), 256, 0, st>>>(a, b, out, n, done);
}
template void launch_sub<double>(const double2*, const double2*, double2*, long long, int,
                                 const int*, cudaStream_t);
template void launch_sub<float>(const float2*, const float2*, float2*, long long, int,
                                const int*, cudaStream_t);
template <class T>
void launch_sub_add_widen(const C<T>* a, const C<T>* b, const C<T>* c, VRef<double> out,
                          long long n, int nrhs, const int* done, cudaStream_t st) {
  HZ_COUNT();
  long long nb = (n + 255) / 256;
  if (nb > 4096) nb = 4096;
  k_sub_add_widen<T><<<dim3((unsigned)nb, nrhs), 256, 0, st>>>(a, b, c, out, n, done);
}
template void launch_sub_add_widen<double>(const double2*, const double2*, const double2*,
                                           VRef<double>, long long, int, const int*,
                                           cudaStream_t);
template void launch_sub_add_widen<float>(const float2*, const float2*, const float2*,
                                          VRef<double>, long long, int, const int*,
                                          cudaStream_t);

void launch_inject(const LevelDev& Lf, const LevelDev& Lc, double* k2c,
                   cudaStream_t st) {
  HZ_COUNT();
  k_inject<<<grid2d(Lc.nx, Lc.ny, 1), dim3(BX, BY), 0, st>>>(Lf, Lc, k2c);
}
void launch_cast_k2(const double* k2d, float* k2f, long long n, cudaStream_t st) {
  HZ_COUNT();
  long long nb = (n + 255) / 256;
  if (nb > 4096) nb = 4096;
  k_cast<<<(unsigned)nb, 256, 0, st>>>(k2d, k2f, n);
}
void launch_dinv(const LevelDev& L, int bc, Shift s, double omega, double2* dd,
                 float2* df, cudaStream_t st) {
  HZ_COUNT();
  k_dinv<<<grid2d(L.nx, L.ny, 1), dim3(BX, BY), 0, st>>>(L, bc, s, omega, dd, df);
}
void launch_dense_assemble(const LevelDev& L, int bc, Shift s, double2* aug,
                           cudaStream_t st) {
  HZ_COUNT();
  const int n = L.nx * L.ny;
  k_dense_assemble<<<(n + 127) / 128, 128, 0, st>>>(L, bc, s, aug);
}
void launch_gauss_jordan(int n, double2* aug, int* err, cudaStream_t st) {
  HZ_COUNT();
  k_gauss_jordan<<<1, 1024, n * sizeof(double2), st>>>(n, aug, err);
}
void launch_extract_inverse(const LevelDev& L, int bc, const double2* aug,
                            double2* md, float2* mf, cudaStream_t st) {
  HZ_COUNT();
  const long long t = (long long)L.nx * L.ny * L.nx * L.ny;
  k_extract<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(L, bc, aug, md, mf);
}

#define HZ_INST(T)                                                              \
  template void launch_helm<T>(const LevelDev&, int, Shift, VRef<T>,            \
                               VRef<T>, C<T>*, int, const int*,                 \
                               cudaStream_t);                                   \
  template void launch_restrict_z<T>(const LevelDev&, const LevelDev&, int,     \
                                     int, VRef<T>, C<T>*, int, const int*,      \
                                     cudaStream_t, double);                     \
  template void launch_prolong_z<T>(const LevelDev&, const LevelDev&, int, int, \
                                    const C<T>*, C<T>*, int, int, const int*,   \
                                    cudaStream_t);                              \
  template void launch_galerkin_fused<T>(const LevelDev&, const LevelDev&, int, \
                                         int, const C<T>*, C<T>*, int,          \
                                         const int*, cudaStream_t);             \
  template void launch_glk<T>(const LevelDev&, int, int, const C<T>*, C<T>*,    \
                              int, const int*, cudaStream_t, double);           \
  template void launch_mask_dirichlet<T>(const LevelDev&, int, C<T>*, int,      \
                                         cudaStream_t);                        \
  template void launch_red_o4<T>(const LevelDev&, int, const C<T>*, C<T>*, int, \
                                 const int*, cudaStream_t);                     \
  template void launch_red_cmpo4<T>(const LevelDev&, int, const C<T>*, C<T>*,   \
                                    int, const int*, cudaStream_t);             \
  template void launch_red_9pt<T>(const LevelDev&, int, const C<T>*, C<T>*,     \
                                  int, const int*, cudaStream_t);               \
  template void launch_red_o6<T>(const LevelDev&, int, const C<T>*, C<T>*, int, \
                                 const int*, cudaStream_t);                     \
  template void launch_probe_extract<T>(const LevelDev&, int, int, int,         \
                                        const double2*, C<T>*, cudaStream_t);   \
  template void launch_stencil_e<T>(const LevelDev&, int, int, const C<T>*,     \
                                    const C<T>*, C<T>*, int, int, const int*,   \
                                    cudaStream_t);                              \
  /* end */

HZ_INST(double)
HZ_INST(float)

template void launch_add_conv<double, double>(VRef<double>, const double2*,
                                              VRef<double>, long long, int,
                                              const int*, cudaStream_t);
template void launch_add_conv<float, float>(VRef<float>, const float2*,
                                            VRef<float>, long long, int,
                                            const int*, cudaStream_t);
template void launch_add_conv<double, float>(VRef<double>, const double2*,
                                             VRef<float>, long long, int,
                                             const int*, cudaStream_t);
template void launch_add_conv<float, double>(VRef<float>, const float2*,
                                             VRef<double>, long long, int,
                                             const int*, cudaStream_t);

}  // namespace hz
