// Matrix-free grid kernels: Helmholtz / CSLP stencils (Sec. 2.1, 3.1, 5.1),
// damped Jacobi, full-weighting restriction and bilinear interpolation
// (Sec. 3.1, 3.2.1), higher-order deflation transfers (Sec. 3.2.1), the
// ReD-Glk coarse stencils (Sec. 5.2.4), the dense coarsest-level solve and
// the setup kernels.  Every kernel serves nrhs right-hand sides (blockIdx.z)
// and skips those flagged done.
#include "hz_common.cuh"

namespace hz {

namespace {

constexpr int BX = 32, BY = 8;

inline dim3 grid2d(int nx, int ny, int nrhs) {
  return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, nrhs);
}

__device__ __forceinline__ bool on_bnd(int i, int j, int nx, int ny) {
  return i == 0 || j == 0 || i == nx - 1 || j == ny - 1;
}

// (M x)(i, j) for an unknown node (i, j): centre 4/h^2 - s k^2, Sommerfeld
// sides add -2 i k / h each, remove the outward neighbour and double the
// opposite one (ghost elimination); Dirichlet rows drop couplings to the
// (fixed zero) boundary nodes.
template <class T>
__device__ __forceinline__ C<T> helm_point(const LevelDev& L, int bc, T sre,
                                           T sim, const C<T>* __restrict__ x,
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
  C<T> acc = cmul(cen, x[id]);
  if (cw != T(0)) acc = rfma(cw, x[id - 1], acc);
  if (ce != T(0)) acc = rfma(ce, x[id + 1], acc);
  if (cs != T(0)) acc = rfma(cs, x[id - nx], acc);
  if (cn != T(0)) acc = rfma(cn, x[id + nx], acc);
  return acc;
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

template <class T>
__global__ void k_jacobi0(LevelDev L, int bc, VRef<T> fin, C<T>* __restrict__ x,
                          const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || (done && done[r])) return;
  const long long n = (long long)L.nx * L.ny, id = (long long)j * L.nx + i;
  if (bc == BC_DIRICHLET && on_bnd(i, j, L.nx, L.ny)) {
    x[r * n + id] = czero<T>();
    return;
  }
  x[r * n + id] = cmul(dinv_of<T>(L)[id], fin.get()[r * n + id]);
}

// fc(I,J) = sum_{a,b in -1..1} (2-|a|)(2-|b|)/16 * (f - M x)(2I+a, 2J+b)
template <class T>
__global__ void k_resid_restrict(LevelDev Lf, LevelDev Lc, int bc, T sre, T sim,
                                 VRef<T> fin, const C<T>* __restrict__ x,
                                 C<T>* __restrict__ fc,
                                 const int* __restrict__ done) {
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (I >= Lc.nx || J >= Lc.ny || (done && done[r])) return;
  const long long nf = (long long)Lf.nx * Lf.ny, nc = (long long)Lc.nx * Lc.ny;
  const long long idc = (long long)J * Lc.nx + I;
  if (bc == BC_DIRICHLET && on_bnd(I, J, Lc.nx, Lc.ny)) {
    fc[r * nc + idc] = czero<T>();
    return;
  }
  const C<T>* f = fin.get() + r * nf;
  const C<T>* xr = x + r * nf;
  C<T> acc = czero<T>();
  for (int b = -1; b <= 1; ++b) {
    const int jf = 2 * J + b;
    if (jf < 0 || jf >= Lf.ny) continue;
    for (int a = -1; a <= 1; ++a) {
      const int jf_i = 2 * I + a;
      if (jf_i < 0 || jf_i >= Lf.nx) continue;
      if (bc == BC_DIRICHLET && on_bnd(jf_i, jf, Lf.nx, Lf.ny)) continue;
      const C<T> res = f[(long long)jf * Lf.nx + jf_i] -
                       helm_point<T>(Lf, bc, sre, sim, xr, jf_i, jf);
      const T w = T((2 - abs(a)) * (2 - abs(b))) * T(0.0625);
      acc = rfma(w, res, acc);
    }
  }
  fc[r * nc + idc] = acc;
}

// bilinear interpolation of xc at fine node (i, j)
template <class T>
__device__ __forceinline__ C<T> interp_bilinear(const LevelDev& Lc,
                                                const C<T>* __restrict__ xc,
                                                int i, int j) {
  const int I0 = i >> 1, J0 = j >> 1;
  const bool ox = i & 1, oy = j & 1;
  const long long b0 = (long long)J0 * Lc.nx + I0;
  C<T> v;
  if (!ox && !oy) return xc[b0];
  if (ox && !oy) {
    v = xc[b0] + xc[b0 + 1];
    return T(0.5) * v;
  }
  if (!ox && oy) {
    v = xc[b0] + xc[b0 + Lc.nx];
    return T(0.5) * v;
  }
  v = (xc[b0] + xc[b0 + 1]) + (xc[b0 + Lc.nx] + xc[b0 + Lc.nx + 1]);
  return T(0.25) * v;
}

template <class T>
__global__ void k_prolong_add(LevelDev Lf, LevelDev Lc, int bc,
                              const C<T>* __restrict__ xc, C<T>* __restrict__ x,
                              const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= Lf.nx || j >= Lf.ny || (done && done[r])) return;
  if (bc == BC_DIRICHLET && on_bnd(i, j, Lf.nx, Lf.ny)) return;
  const long long nf = (long long)Lf.nx * Lf.ny, nc = (long long)Lc.nx * Lc.ny;
  const long long id = (long long)j * Lf.nx + i;
  x[r * nf + id] = x[r * nf + id] + interp_bilinear<T>(Lc, xc + r * nc, i, j);
}

template <class T>
__global__ void k_smooth(LevelDev L, int bc, T sre, T sim, VRef<T> fin,
                         const C<T>* __restrict__ x, C<T>* __restrict__ xo,
                         const int* __restrict__ done) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || (done && done[r])) return;
  const long long n = (long long)L.nx * L.ny, id = (long long)j * L.nx + i;
  if (bc == BC_DIRICHLET && on_bnd(i, j, L.nx, L.ny)) {
    xo[r * n + id] = czero<T>();
    return;
  }
  const C<T>* xr = x + r * n;
  const C<T> res = fin.get()[r * n + id] - helm_point<T>(L, bc, sre, sim, xr, i, j);
  xo[r * n + id] = cfma(dinv_of<T>(L)[id], res, xr[id]);
}

// 1-D weights of Z^T: bilinear [1 2 1]/2 at offsets -1..1, higher-order
// [1 4 6 4 1]/8 at offsets -2..2; R_Z = Z^T / 4 is their tensor product / 4.
template <class T>
__global__ void k_restrict_z(LevelDev Lf, LevelDev Lc, int bc, int zk,
                             VRef<T> fin, C<T>* __restrict__ coarse,
                             const int* __restrict__ done) {
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
  coarse[r * nc + idc] = acc;
}

// 1-D interpolation weights of a fine node: (coarse index, weight) pairs.
template <class T>
__device__ __forceinline__ int z1d(int zk, int i, int nc, int* idx, T* w) {
  int k = 0;
  if (i & 1) {
    idx[0] = i >> 1; w[0] = T(0.5);
    idx[1] = (i >> 1) + 1; w[1] = T(0.5);
    return 2;
  }
  const int I = i >> 1;
  if (zk != ZK_HO) {
    idx[0] = I; w[0] = T(1);
    return 1;
  }
  if (I - 1 >= 0) { idx[k] = I - 1; w[k] = T(0.125); ++k; }
  idx[k] = I; w[k] = T(0.75); ++k;
  if (I + 1 < nc) { idx[k] = I + 1; w[k] = T(0.125); ++k; }
  return k;
}

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
  int ix[3], iy[3];
  T wx[3], wy[3];
  const int nxk = z1d<T>(zk, i, Lc.nx, ix, wx);
  const int nyk = z1d<T>(zk, j, Lc.ny, iy, wy);
  const C<T>* c = coarse + r * nc;
  C<T> acc = czero<T>();
  for (int b = 0; b < nyk; ++b) {
    for (int a = 0; a < nxk; ++a) {
      if (bc == BC_DIRICHLET && on_bnd(ix[a], iy[b], Lc.nx, Lc.ny)) continue;
      acc = rfma(wx[a] * wy[b], c[(long long)iy[b] * Lc.nx + ix[a]], acc);
    }
  }
  fine[r * nf + id] = add ? fine[r * nf + id] + acc : acc;
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
// the average of reaching them through x first and through y first, with
// the wavenumber of a ghost node taken as zero.
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
  if (bc == BC_SOMMERFELD) {  // ghost k = 0: the rule returns the inner value
    ox = gyv(ii, j);
    oy = gxv(i, jj);
  } else {
    ox = T(2) * gyv(bi, j) - gyv(ii, j);
    oy = T(2) * gxv(i, bj) - gxv(i, jj);
  }
  return T(0.5) * (ox + oy);
}

template <class T>
__global__ void k_glk(LevelDev L, int bc, int variant, const C<T>* __restrict__ x,
                      C<T>* __restrict__ y, const int* __restrict__ done) {
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
  y[r * n + id] = acc;
}

template <class T>
__global__ void k_mask_dirichlet(LevelDev L, C<T>* __restrict__ x) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  const int r = blockIdx.z;
  if (i >= L.nx || j >= L.ny || !on_bnd(i, j, L.nx, L.ny)) return;
  x[(long long)r * L.nx * L.ny + (long long)j * L.nx + i] = czero<T>();
}

template <class T>
__global__ void k_dense_mv(int n, const C<T>* __restrict__ minv, VRef<T> fin,
                           C<T>* __restrict__ x, const int* __restrict__ done) {
  extern __shared__ unsigned char smraw[];
  C<T>* fs = reinterpret_cast<C<T>*>(smraw);
  const int r = blockIdx.y;
  if (done && done[r]) return;
  const C<T>* f = fin.get();
  for (int c = threadIdx.x; c < n; c += blockDim.x) fs[c] = f[(long long)r * n + c];
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const C<T>* mr = minv + (long long)row * n;
  C<T> acc = czero<T>();
  for (int c = 0; c < n; ++c) acc = cfma(mr[c], fs[c], acc);
  x[(long long)r * n + row] = acc;
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
void launch_jacobi0(const LevelDev& L, int bc, VRef<T> f, C<T>* x, int nrhs,
                    const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_jacobi0<T><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(L, bc, f, x, done);
}
template <class T>
void launch_resid_restrict(const LevelDev& Lf, const LevelDev& Lc, int bc,
                           Shift s, VRef<T> f, const C<T>* x, C<T>* fc,
                           int nrhs, const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_resid_restrict<T><<<grid2d(Lc.nx, Lc.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, (T)s.re, (T)s.im, f, x, fc, done);
}
template <class T>
void launch_prolong_add(const LevelDev& Lf, const LevelDev& Lc, int bc,
                        const C<T>* xc, C<T>* x, int nrhs, const int* done,
                        cudaStream_t st) {
  HZ_COUNT();
  k_prolong_add<T><<<grid2d(Lf.nx, Lf.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, xc, x, done);
}
template <class T>
void launch_smooth(const LevelDev& L, int bc, Shift s, VRef<T> f,
                   const C<T>* x, C<T>* xo, int nrhs, const int* done,
                   cudaStream_t st) {
  HZ_COUNT();
  k_smooth<T><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(
      L, bc, (T)s.re, (T)s.im, f, x, xo, done);
}
template <class T>
void launch_restrict_z(const LevelDev& Lf, const LevelDev& Lc, int bc, int zk,
                       VRef<T> fine, C<T>* coarse, int nrhs, const int* done,
                       cudaStream_t st) {
  HZ_COUNT();
  k_restrict_z<T><<<grid2d(Lc.nx, Lc.ny, nrhs), dim3(BX, BY), 0, st>>>(
      Lf, Lc, bc, zk, fine, coarse, done);
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
void launch_glk(const LevelDev& L, int bc, int variant, const C<T>* x, C<T>* y,
                int nrhs, const int* done, cudaStream_t st) {
  HZ_COUNT();
  k_glk<T><<<grid2d(L.nx, L.ny, nrhs), dim3(BX, BY), 0, st>>>(L, bc, variant, x,
                                                               y, done);
}
template <class T>
void launch_dense_mv(int n, const C<T>* minv, VRef<T> f, C<T>* x, int nrhs,
                     const int* done, cudaStream_t st) {
  HZ_COUNT();
  const int nt = 128;
  k_dense_mv<T><<<dim3((n + nt - 1) / nt, nrhs), nt, n * sizeof(C<T>), st>>>(
      n, minv, f, x, done);
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
  template void launch_jacobi0<T>(const LevelDev&, int, VRef<T>, C<T>*, int,    \
                                  const int*, cudaStream_t);                    \
  template void launch_resid_restrict<T>(const LevelDev&, const LevelDev&, int, \
                                         Shift, VRef<T>, const C<T>*, C<T>*,    \
                                         int, const int*, cudaStream_t);        \
  template void launch_prolong_add<T>(const LevelDev&, const LevelDev&, int,    \
                                      const C<T>*, C<T>*, int, const int*,      \
                                      cudaStream_t);                            \
  template void launch_smooth<T>(const LevelDev&, int, Shift, VRef<T>,          \
                                 const C<T>*, C<T>*, int, const int*,           \
                                 cudaStream_t);                                 \
  template void launch_restrict_z<T>(const LevelDev&, const LevelDev&, int,     \
                                     int, VRef<T>, C<T>*, int, const int*,      \
                                     cudaStream_t);                             \
  template void launch_prolong_z<T>(const LevelDev&, const LevelDev&, int, int, \
                                    const C<T>*, C<T>*, int, int, const int*,   \
                                    cudaStream_t);                              \
  template void launch_glk<T>(const LevelDev&, int, int, const C<T>*, C<T>*,    \
                              int, const int*, cudaStream_t);                   \
  template void launch_mask_dirichlet<T>(const LevelDev&, int, C<T>*, int,      \
                                         cudaStream_t);                        \
  template void launch_dense_mv<T>(int, const C<T>*, VRef<T>, C<T>*, int,       \
                                   const int*, cudaStream_t);

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
